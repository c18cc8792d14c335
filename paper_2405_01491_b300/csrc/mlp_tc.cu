// Tensor-core (tcgen05) BF16 form of the per-element networks (section II.B) with FP32 accumulation.
//
// Same products as the FP32 form (mlp_simt.cu), on 128 x NT tiles of tc_gemm.cuh:
//   L1  h1 = CELU(aev W1cat^T + b1)              NT = 256, N = M*256, K = 1008 (two-SM tiles, tc_pair.cuh)
//   L2  h2 = CELU(h1_m W2^T + b2)                NT = 192 per member
//   L3  g3 = (1/M) w4 CELU'(z3), y_m = h3 . w4   NT = 160 per member (whole row in one tile)
//   L3' g2 = (g3_m W3) * CELU'(z2)               NT = 192
//   (bf16 and split forms: L3 and L3' are one kernel, tc_fused.cuh, with g3 kept in TMEM)
//   L2' g1 = (g2_m W2) * CELU'(z1)               NT = 256
//   L1' dE/dAEV = g1 W1cat                       NT = 256, N = 1008, K = M*256, fp32 out (two-SM tiles)
// Activations between layers are bf16 in HBM; operands reach shared memory by TMA (3-D tensor maps
// whose middle coordinate selects the member, so each member's K range ends in zero fill).  The split
// (FP32X3) products stage hi and lo of both operands per K chunk and issue hi*hi + hi*lo + lo*hi from
// one stage, so each operand tile crosses L2 once per tile instead of twice.
//
// FP8 form: the same six products with e4m3 operands (tcgen05 kind::f8f6f4) and per-layer scaling.
// Each weight block (member, element, layer) carries the scale amax / 448 (W1^T one per element, as
// its K runs over all members); each activation tensor (AEV, h1, h2, g3, g2, g1) one scale per
// layer, 2 amax / 448 from a calibration evaluation in FP32 (x2 headroom; conversions saturate).  The
// epilogue multiplies the fp32 accumulator by a_scale * b_scale and writes its output as
// e4m3(x / out_scale).
#include <cudaTypedefs.h>

#include <cmath>
#include <cstring>
#include <type_traits>
#include <vector>

#include "tc_fused.cuh"
#include "tc_gemm.cuh"
#include "tc_pair.cuh"

namespace fnn {

void free_train_tc(void *p);

namespace {

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

// 3-D bf16 tensor map: dims (d0 innermost, d1, d2), byte strides of d1 and d2, box (b0, b1, b2), 128-byte swizzle
bool encode3d(CUtensorMap *m, const void *base, uint64_t d0, uint64_t d1, uint64_t d2, uint64_t s1, uint64_t s2,
              uint32_t b0, uint32_t b1, uint32_t b2, CUtensorMapDataType dt = CU_TENSOR_MAP_DATA_TYPE_BFLOAT16,
              CUtensorMapSwizzle sw = CU_TENSOR_MAP_SWIZZLE_128B) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = encode_fn();
  if (!enc) return false;
  cuuint64_t dims[3] = {d0, d1, d2};
  cuuint64_t str[2] = {s1, s2};
  cuuint32_t box[3] = {b0, b1, b2}, es[3] = {1, 1, 1};
  return enc(m, dt, 3, const_cast<void *>(base), dims, str, box, es,
             CU_TENSOR_MAP_INTERLEAVE_NONE, sw, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// One half (hi or lo) of the bf16 operands: the BF16 form uses the hi half only (bf16(x) is exactly the
// hi term of the split), the three-term FP32 form uses both.
struct Half {
  __nv_bfloat16 *W1 = nullptr, *W1T = nullptr, *W2 = nullptr, *W2T = nullptr, *W3 = nullptr, *W3T = nullptr;
  CUtensorMap mW1, mW1T, mW2, mW2T, mW3, mW3T;
  __nv_bfloat16 *aev = nullptr, *h1 = nullptr, *h2 = nullptr, *g3 = nullptr, *g2 = nullptr, *g1 = nullptr;
  CUtensorMap mAev, mH1, mH2, mG3, mG2, mG1;   // operand maps (128-byte rows, swizzled)
  CUtensorMap eH1, eH2, eG3, eG2, eG1;         // epilogue maps: 32-row x 16-column pieces, unswizzled
  // 64-byte-row (64-byte swizzle) operand maps (the split first-layer input gradient, the fused third layer)
  CUtensorMap qW1T, qG1, qW3, qW3T, qH2;
  // weights with 64-row boxes: the column strips of a product's partial last wave, the two-SM tiles' halves
  CUtensorMap sW1, sW2, sW2T, sW1T;
  // 64 rows x 64 features (MN-major operands of the weight gradients)
  CUtensorMap wAev, wH1, wH2;
};

// e4m3 operands of the FP8 form and their scales
struct F8 {
  uint8_t *wbuf = nullptr;
  uint8_t *W1 = nullptr, *W1T = nullptr, *W2 = nullptr, *W2T = nullptr, *W3 = nullptr, *W3T = nullptr;
  CUtensorMap mW1, mW1T, mW2, mW2T, mW3, mW3T;
  CUtensorMap sW1;           // W1 with 64-row boxes (the two-SM first layer's weight halves)
  float *wscale = nullptr;   // device [6][M*7] in the order W1, W1T, W2, W2T, W3, W3T; W1T per element only
  uint8_t *abuf = nullptr;
  size_t rows = 0;
  uint8_t *aev = nullptr, *h1 = nullptr, *h2 = nullptr, *g3 = nullptr, *g2 = nullptr, *g1 = nullptr;
  CUtensorMap mAev, mH1, mH2, mG3, mG2, mG1;
  CUtensorMap eH1, eH2, eG3, eG2, eG1;
  unsigned *amax = nullptr;  // device [6] calibration maxima (float bits)
  float act[6] = {1, 1, 1, 1, 1, 1};  // scales of aev, h1, h2, g3, g2, g1
  bool calibrated = false;
};

struct TcState {
  int M = 0;
  __nv_bfloat16 *wbuf = nullptr;
  __nv_bfloat16 *abuf = nullptr;
  size_t rows = 0;
  Half h[2];   // [0] hi, [1] lo
  F8 f8;
  // fp32 dE/dAEV [rows][1008] as the input-gradient product's output map (32-row x 8-column boxes)
  CUtensorMap mGaev;
  const float *gaev_for = nullptr;
  size_t gaev_rows = 0;
  void *train = nullptr;   // BF16 training buffers (tc_param_grads)
};

TcState *state(fnn_ctx *ctx) {
  if (!ctx->w.tc) ctx->w.tc = new TcState();
  return static_cast<TcState *>(ctx->w.tc);
}

// the output map of ws.gaev, re-encoded when the workspace moved
static const CUtensorMap *gaev_map(fnn_ctx *ctx, TcState *t) {
  if (t->gaev_for != ctx->ws.gaev || t->gaev_rows != ctx->ws.rows) {
    if (!encode3d(&t->mGaev, ctx->ws.gaev, NAEV, 1, ctx->ws.rows, NAEV * 4, NAEV * 4, 8, 1, 32,
                  CU_TENSOR_MAP_DATA_TYPE_FLOAT32, CU_TENSOR_MAP_SWIZZLE_NONE))
      return nullptr;
    t->gaev_for = ctx->ws.gaev;
    t->gaev_rows = ctx->ws.rows;
  }
  return &t->mGaev;
}

// Operand, output and aux tensor maps of one product (lo = the split's low halves; unused ones may
// repeat any valid map).
struct Maps {
  const CUtensorMap *A, *B, *A_lo, *B_lo, *O, *O_lo, *X, *X_lo;
  const CUtensorMap *Bs = nullptr, *Bs_lo = nullptr;   // B with strip-high boxes (tail column strips)
};

// tail-tile zeroing: ZT_PARTS blocks of 64 threads per 128-row tile, 16-byte stores
constexpr int ZT_PARTS = 8;

// fused third layer (tc_fused.cuh): persistent over the (row tile, member) grid
template <int MODE, int KB>
fnn_status launch_l3_pair(fnn_ctx *ctx, const char *name, const CUtensorMap *const maps[10], tc::L3Args a,
                          cudaStream_t s) {
  const long long T = (long long)a.n_rowtiles * a.n_members;
  if (T == 0) return FNN_OK;
  dim3 grid((unsigned)(T < ctx->num_sms ? T : ctx->num_sms));
  static bool attr_set = false;
  const size_t sm = tc::l3_smem_bytes<MODE, KB>();
  if (!attr_set) {
    FNN_CUDA_TRY(ctx, cudaFuncSetAttribute(tc::k_l3_pair<MODE, KB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    attr_set = true;
  }
  FNN_KERNEL(ctx, name, s);
  tc::k_l3_pair<MODE, KB><<<grid, tc::THREADS, sm, s>>>(*maps[0], *maps[1], *maps[2], *maps[3], *maps[4], *maps[5],
                                                    *maps[6], *maps[7], *maps[8], *maps[9], a);
  return check_launch(ctx, name);
}

template <int NT, int EPI, int MODE, bool QUAD = false, int KB = tc::BKB>
fnn_status launch(fnn_ctx *ctx, const char *name, const Maps &mp, tc::Args a, dim3 tiles, cudaStream_t s) {
  // persistent launch: at most one CTA per SM over the (n tile, row tile, member) grid; a launch whose partial
  // wave is split (K parts or column strips) takes every SM, the split's parts being spread over the grid
  a.n_ntiles = (int)tiles.x;
  a.n_rowtiles = (int)tiles.y;
  a.n_members = (int)tiles.z;
  const long long T = (long long)tiles.x * tiles.y * tiles.z;
  dim3 grid((unsigned)(T < ctx->num_sms && !a.tail_split && !a.tail_nsplit ? T : ctx->num_sms));
  static bool attr_set = false;
  const size_t sm = tc::smem_bytes<NT, EPI, MODE, QUAD, KB>();
  if (!attr_set) {
    FNN_CUDA_TRY(ctx, cudaFuncSetAttribute(tc::k_umma<NT, EPI, MODE, QUAD, KB>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    attr_set = true;
  }
  FNN_KERNEL(ctx, name, s);
  tc::k_umma<NT, EPI, MODE, QUAD, KB><<<grid, tc::THREADS, sm, s>>>(
      *mp.A, *mp.B, *mp.A_lo, *mp.B_lo, *mp.O, *mp.O_lo, *mp.X, *mp.X_lo, mp.Bs ? *mp.Bs : *mp.B,
      mp.Bs_lo ? *mp.Bs_lo : *mp.B_lo, a);
  return check_launch(ctx, name);
}

// The two-SM first-layer forward (tc_pair.cuh): clusters of two CTAs, persistent over the (member, row-tile
// pair) items; as many clusters as fit at once, at most one CTA per SM.
template <int MODE, int EPI = tc::EPI_BIAS_CELU>
fnn_status pair_launch_config(fnn_ctx *ctx, cudaLaunchConfig_t &cfg, cudaLaunchAttribute *attr, int &ncl,
                              cudaStream_t s) {
  const size_t sm = tc::pair_smem_bytes<MODE, EPI>();
  static bool attr_set = false;
  static int max_cl = 0;
  cfg = cudaLaunchConfig_t{};
  cfg.blockDim = dim3(tc::THREADS);
  cfg.dynamicSmemBytes = sm;
  cfg.stream = s;
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = 2;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (!attr_set) {
    FNN_CUDA_TRY(ctx, cudaFuncSetAttribute(tc::k_umma_pair<MODE, EPI>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)sm));
    cfg.gridDim = dim3((unsigned)(ctx->num_sms & ~1));
    FNN_CUDA_TRY(ctx, cudaOccupancyMaxActiveClusters(&max_cl, tc::k_umma_pair<MODE, EPI>, &cfg));
    attr_set = true;
  }
  if (max_cl < 1) {
    ctx->last_error = "two-SM first layer: no cluster of two CTAs fits on the device";
    return FNN_E_CUDA;
  }
  ncl = max_cl < ctx->num_sms / 2 ? max_cl : ctx->num_sms / 2;
  cfg.gridDim = dim3((unsigned)(2 * ncl));
  return FNN_OK;
}
template <int MODE, int EPI = tc::EPI_BIAS_CELU>
fnn_status launch_pair(fnn_ctx *ctx, const char *name, const CUtensorMap *A, const CUtensorMap *A_lo,
                       const CUtensorMap *B, const CUtensorMap *B_lo, const CUtensorMap *O, const CUtensorMap *O_lo,
                       const tc::PairArgs &a, cudaStream_t s) {
  cudaLaunchConfig_t cfg;
  cudaLaunchAttribute attr[1];
  int ncl;
  fnn_status st;
  if ((st = pair_launch_config<MODE, EPI>(ctx, cfg, attr, ncl, s))) return st;
  FNN_KERNEL(ctx, name, s);
  FNN_CUDA_TRY(ctx, cudaLaunchKernelEx(&cfg, tc::k_umma_pair<MODE, EPI>, *A, *A_lo, *B, *B_lo, *O, *O_lo, a));
  return check_launch(ctx, name);
}

// zero the tiles of the pair schedule's partial wave that a tail-split fp32 launch on ncl clusters adds its
// K parts into (tc::pair_tail_sched): ZT_PARTS blocks of 64 threads per row tile of each tail item
__global__ void __launch_bounds__(64) k_zero_tail_pair(const int32_t *meta, int n_nt, int ncl, int nkb, int N,
                                                       float *out, long long ldo) {
  int seg[NE + 1];
  for (int e = 0; e <= NE; e++) seg[e] = meta[META_SEG + e];
  int T = 0;
  for (int e = 0; e < NE; e++) T += (seg[e + 1] / tc::BM - seg[e] / tc::BM + 1) / 2;
  T *= n_nt;
  const tc::PairTail ts = tc::pair_tail_sched(T, ncl, nkb);
  const int item = (int)blockIdx.x / (2 * ZT_PARTS), half = ((int)blockIdx.x / ZT_PARTS) & 1,
            part = (int)blockIdx.x % ZT_PARTS;
  if (item >= ts.R) return;
  int nt, rt0, e;
  bool two;
  if (!tc::pair_item(seg, n_nt, ts.W * ncl + item, nt, rt0, e, two) || (half && !two)) return;
  const int rt = rt0 + half, c0 = nt * tc::PAIR_NT, n4 = min(tc::PAIR_NT, N - c0) / 4;
  const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
  for (int rr = 0; rr < tc::BM / ZT_PARTS; rr++) {
    float *row = out + ((long long)rt * tc::BM + part * (tc::BM / ZT_PARTS) + rr) * ldo + c0;
    for (int c4 = threadIdx.x; c4 < n4; c4 += 64) reinterpret_cast<float4 *>(row)[c4] = z;
  }
}

// the split with four-tile stages (hi and lo of both operands per K chunk) where quad is set
// (and, where mp64 is given, 64-byte operand rows: twice the stages for the same bytes in flight)
template <int NT, int EPI, int MODE>
fnn_status launch_q(bool quad, fnn_ctx *ctx, const char *name, const Maps &mp, const Maps *mp64, tc::Args a,
                    dim3 tiles, cudaStream_t s) {
  if constexpr (MODE == tc::MODE_SPLIT) {
    if (quad && mp64) return launch<NT, EPI, MODE, true, 64>(ctx, name, *mp64, a, tiles, s);
    if (quad) return launch<NT, EPI, MODE, true>(ctx, name, mp, a, tiles, s);
  }
  return launch<NT, EPI, MODE, false>(ctx, name, mp, a, tiles, s);
}

}  // namespace

void free_tc(fnn_ctx *ctx) {
  TcState *t = static_cast<TcState *>(ctx->w.tc);
  if (!t) return;
  if (t->wbuf) cudaFree(t->wbuf);
  if (t->abuf) cudaFree(t->abuf);
  if (t->f8.wbuf) cudaFree(t->f8.wbuf);
  if (t->f8.wscale) cudaFree(t->f8.wscale);
  if (t->f8.abuf) cudaFree(t->f8.abuf);
  if (t->f8.amax) cudaFree(t->f8.amax);
  free_train_tc(t->train);
  delete t;
  ctx->w.tc = nullptr;
}

// e4m3 copies of the six layer matrices, each (member, element) block scaled by its amax / 448
static fnn_status upload_f8_weights(fnn_ctx *ctx, TcState *t, const float *const src[6], const size_t len[6]) {
  F8 &f = t->f8;
  const int M = t->M;
  if (f.wbuf) cudaFree(f.wbuf);
  if (f.wscale) cudaFree(f.wscale);
  f.wbuf = nullptr;
  f.wscale = nullptr;
  f.calibrated = false;
  size_t total = 0, off[6];
  for (int k = 0; k < 6; k++) {
    off[k] = total;
    total += len[k];
  }
  std::vector<uint8_t> q(total);
  std::vector<float> scale((size_t)6 * M * NE, 1.f);
  // block b of matrix k: element e, member m; returns the indices of its entries through a visitor
  auto visit = [&](int k, int m, int e, auto fn) {
    const float *w = src[k];
    if (k == 0) {          // W1cat [7][M*256][1008]: rows m*256.. of element e
      const size_t b = ((size_t)e * M + m) * H1 * NAEV;
      for (size_t i = 0; i < (size_t)H1 * NAEV; i++) fn(b + i, w[b + i]);
    } else if (k == 1) {   // W1Tcat [7][1008][M*256]: all members of element e
      const size_t b = (size_t)e * NAEV * M * H1;
      for (size_t i = 0; i < (size_t)NAEV * M * H1; i++) fn(b + i, w[b + i]);
    } else {               // [M][7][out][in]
      const size_t n = (k < 4) ? (size_t)H2 * H1 : (size_t)H3 * H2;
      const size_t b = ((size_t)m * NE + e) * n;
      for (size_t i = 0; i < n; i++) fn(b + i, w[b + i]);
    }
  };
  for (int k = 0; k < 6; k++)
    for (int m = 0; m < (k == 1 ? 1 : M); m++)
      for (int e = 0; e < NE; e++) {
        float amax = 0.f;
        visit(k, m, e, [&](size_t, float x) { amax = fmaxf(amax, fabsf(x)); });
        const float sc = amax > 0.f ? amax / 448.f : 1.f;
        scale[(size_t)k * M * NE + (size_t)m * NE + e] = sc;
        const float inv = 1.f / sc;
        visit(k, m, e, [&](size_t i, float x) { q[off[k] + i] = __nv_cvt_float_to_fp8(x * inv, __NV_SATFINITE, __NV_E4M3); });
      }
  if (cudaMalloc(&f.wbuf, total) != cudaSuccess || cudaMalloc(&f.wscale, scale.size() * sizeof(float)) != cudaSuccess) {
    cudaGetLastError();
    ctx->last_error = "cudaMalloc failed for fp8 weights";
    return FNN_E_OOM;
  }
  FNN_CUDA_TRY(ctx, cudaMemcpy(f.wbuf, q.data(), total, cudaMemcpyHostToDevice));
  FNN_CUDA_TRY(ctx, cudaMemcpy(f.wscale, scale.data(), scale.size() * sizeof(float), cudaMemcpyHostToDevice));
  f.W1 = f.wbuf + off[0]; f.W1T = f.wbuf + off[1]; f.W2 = f.wbuf + off[2];
  f.W2T = f.wbuf + off[3]; f.W3 = f.wbuf + off[4]; f.W3T = f.wbuf + off[5];
  const uint64_t G = (uint64_t)M * NE;
  const CUtensorMapDataType U8 = CU_TENSOR_MAP_DATA_TYPE_UINT8;
  bool ok = encode3d(&f.mW1, f.W1, NAEV, (uint64_t)M * H1, NE, NAEV, (uint64_t)M * H1 * NAEV, 128, 256, 1, U8) &&
            encode3d(&f.sW1, f.W1, NAEV, (uint64_t)M * H1, NE, NAEV, (uint64_t)M * H1 * NAEV, 128, 64, 1, U8) &&
            encode3d(&f.mW1T, f.W1T, (uint64_t)M * H1, NAEV, NE, (uint64_t)M * H1, (uint64_t)NAEV * M * H1, 128, 256,
                     1, U8) &&
            encode3d(&f.mW2, f.W2, H1, H2, G, H1, (uint64_t)H2 * H1, 128, H2, 1, U8) &&
            encode3d(&f.mW2T, f.W2T, H2, H1, G, H2, (uint64_t)H1 * H2, 128, H1, 1, U8) &&
            encode3d(&f.mW3, f.W3, H2, H3, G, H2, (uint64_t)H3 * H2, 128, H3, 1, U8) &&
            encode3d(&f.mW3T, f.W3T, H3, H2, G, H3, (uint64_t)H2 * H3, 128, H2, 1, U8);
  if (!ok) {
    ctx->last_error = "cuTensorMapEncodeTiled failed for the fp8 weight maps";
    return FNN_E_CUDA;
  }
  return FNN_OK;
}

// bf16 hi and lo halves of the layer matrices in the FP32 form's layouts (host arrays in those layouts):
// hi = bf16(w), lo = bf16(w - hi)
fnn_status upload_tc_weights(fnn_ctx *ctx, int M, const float *W1cat, const float *W1Tcat, const float *W2,
                             const float *W2T, const float *W3, const float *W3T) {
  TcState *t = state(ctx);
  if (t->wbuf) cudaFree(t->wbuf);
  t->wbuf = nullptr;
  const size_t n1 = (size_t)NE * M * H1 * NAEV, n2 = (size_t)M * NE * H2 * H1, n3 = (size_t)M * NE * H3 * H2;
  const size_t half = 2 * (n1 + n2 + n3);
  std::vector<__nv_bfloat16> h(2 * half);
  const float *src[6] = {W1cat, W1Tcat, W2, W2T, W3, W3T};
  const size_t len[6] = {n1, n1, n2, n2, n3, n3};
  size_t off[6], o = 0;
  for (int k = 0; k < 6; k++) {
    off[k] = o;
    for (size_t i = 0; i < len[k]; i++) {
      const __nv_bfloat16 hi = __float2bfloat16(src[k][i]);
      h[o + i] = hi;
      h[half + o + i] = __float2bfloat16(src[k][i] - __bfloat162float(hi));
    }
    o += len[k];
  }
  if (cudaMalloc(&t->wbuf, 2 * half * sizeof(__nv_bfloat16)) != cudaSuccess) {
    cudaGetLastError();
    ctx->last_error = "cudaMalloc failed for bf16 weights";
    return FNN_E_OOM;
  }
  FNN_CUDA_TRY(ctx, cudaMemcpy(t->wbuf, h.data(), 2 * half * sizeof(__nv_bfloat16), cudaMemcpyHostToDevice));
  t->M = M;
  const uint64_t G = (uint64_t)M * NE;
  for (int q = 0; q < 2; q++) {
    Half &H = t->h[q];
    __nv_bfloat16 *base = t->wbuf + q * half;
    H.W1 = base + off[0]; H.W1T = base + off[1]; H.W2 = base + off[2];
    H.W2T = base + off[3]; H.W3 = base + off[4]; H.W3T = base + off[5];
    bool ok =
        encode3d(&H.mW1, H.W1, NAEV, (uint64_t)M * H1, NE, NAEV * 2, (uint64_t)M * H1 * NAEV * 2, 64, 256, 1) &&
        encode3d(&H.mW1T, H.W1T, (uint64_t)M * H1, NAEV, NE, (uint64_t)M * H1 * 2, (uint64_t)NAEV * M * H1 * 2, 64, 256,
                 1) &&
        encode3d(&H.mW2, H.W2, H1, H2, G, H1 * 2, (uint64_t)H2 * H1 * 2, 64, H2, 1) &&
        encode3d(&H.mW2T, H.W2T, H2, H1, G, H2 * 2, (uint64_t)H1 * H2 * 2, 64, H1, 1) &&
        encode3d(&H.mW3, H.W3, H2, H3, G, H2 * 2, (uint64_t)H3 * H2 * 2, 64, H3, 1) &&
        encode3d(&H.mW3T, H.W3T, H3, H2, G, H3 * 2, (uint64_t)H2 * H3 * 2, 64, H2, 1);
    const CUtensorMapDataType BF = CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
    const CUtensorMapSwizzle S64 = CU_TENSOR_MAP_SWIZZLE_64B;
    ok = ok && encode3d(&H.qW1T, H.W1T, (uint64_t)M * H1, NAEV, NE, (uint64_t)M * H1 * 2, (uint64_t)NAEV * M * H1 * 2,
                        32, 256, 1, BF, S64) &&
         encode3d(&H.qW3, H.W3, H2, H3, G, H2 * 2, (uint64_t)H3 * H2 * 2, 32, H3, 1, BF, S64) &&
         encode3d(&H.qW3T, H.W3T, H3, H2, G, H3 * 2, (uint64_t)H2 * H3 * 2, 32, H2, 1, BF, S64) &&
         encode3d(&H.sW1, H.W1, NAEV, (uint64_t)M * H1, NE, NAEV * 2, (uint64_t)M * H1 * NAEV * 2, 64, 64, 1) &&
         encode3d(&H.sW1T, H.W1T, (uint64_t)M * H1, NAEV, NE, (uint64_t)M * H1 * 2, (uint64_t)NAEV * M * H1 * 2, 64, 64,
                  1) &&
         encode3d(&H.sW2, H.W2, H1, H2, G, H1 * 2, (uint64_t)H2 * H1 * 2, 64, 64, 1) &&
         encode3d(&H.sW2T, H.W2T, H2, H1, G, H2 * 2, (uint64_t)H1 * H2 * 2, 64, 64, 1);
    if (!ok) {
      ctx->last_error = "cuTensorMapEncodeTiled failed for the weight maps";
      return FNN_E_CUDA;
    }
  }
  return upload_f8_weights(ctx, t, src, len);
}

static fnn_status tc_workspace(fnn_ctx *ctx, size_t rows, int halves) {
  TcState *t = state(ctx);
  const int M = t->M;
  const bool have = t->abuf && rows <= t->rows && (halves == 1 || t->h[1].aev);
  if (have) return FNN_OK;
  ctx->gen++;
  rows = rows + rows / 8;
  if (t->abuf) cudaFree(t->abuf);
  t->abuf = nullptr;
  t->h[1].aev = nullptr;
  const size_t per_row = NAEV + (size_t)M * (H1 + H2 + H3 + H2 + H1);
  if (cudaMalloc(&t->abuf, 2 * rows * per_row * sizeof(__nv_bfloat16)) != cudaSuccess) {
    cudaGetLastError();
    ctx->last_error = "cudaMalloc failed for bf16 activations";
    return FNN_E_OOM;
  }
  t->rows = rows;
  const uint64_t R = rows;
  for (int q = 0; q < 2; q++) {
    Half &H = t->h[q];
    __nv_bfloat16 *p = t->abuf + q * rows * per_row;
    H.aev = p; p += rows * NAEV;
    H.h1 = p; p += rows * M * H1;
    H.h2 = p; p += rows * M * H2;
    H.g3 = p; p += rows * M * H3;
    H.g2 = p; p += rows * M * H2;
    H.g1 = p;
    bool ok = encode3d(&H.mAev, H.aev, NAEV, 1, R, NAEV * 2, NAEV * 2, 64, 1, 128) &&
              encode3d(&H.mH1, H.h1, H1, M, R, H1 * 2, (uint64_t)M * H1 * 2, 64, 1, 128) &&
              encode3d(&H.mH2, H.h2, H2, M, R, H2 * 2, (uint64_t)M * H2 * 2, 64, 1, 128) &&
              encode3d(&H.mG3, H.g3, H3, M, R, H3 * 2, (uint64_t)M * H3 * 2, 64, 1, 128) &&
              encode3d(&H.mG2, H.g2, H2, M, R, H2 * 2, (uint64_t)M * H2 * 2, 64, 1, 128) &&
              encode3d(&H.mG1, H.g1, (uint64_t)M * H1, 1, R, (uint64_t)M * H1 * 2, (uint64_t)M * H1 * 2, 64, 1, 128);
    const CUtensorMapDataType BF = CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
    const CUtensorMapSwizzle NS = CU_TENSOR_MAP_SWIZZLE_NONE, S64 = CU_TENSOR_MAP_SWIZZLE_64B;
    ok = ok && encode3d(&H.qG1, H.g1, (uint64_t)M * H1, 1, R, (uint64_t)M * H1 * 2, (uint64_t)M * H1 * 2, 32, 1, 128,
                        BF, S64) &&
         encode3d(&H.qH2, H.h2, H2, M, R, H2 * 2, (uint64_t)M * H2 * 2, 32, 1, 128, BF, S64) &&
         encode3d(&H.wAev, H.aev, NAEV, 1, R, NAEV * 2, NAEV * 2, 64, 1, 64) &&
         encode3d(&H.wH1, H.h1, H1, M, R, H1 * 2, (uint64_t)M * H1 * 2, 64, 1, 64) &&
         encode3d(&H.wH2, H.h2, H2, M, R, H2 * 2, (uint64_t)M * H2 * 2, 64, 1, 64);
    ok = ok && encode3d(&H.eH1, H.h1, H1, M, R, H1 * 2, (uint64_t)M * H1 * 2, 16, 1, 32, BF, NS) &&
         encode3d(&H.eH2, H.h2, H2, M, R, H2 * 2, (uint64_t)M * H2 * 2, 16, 1, 32, BF, NS) &&
         encode3d(&H.eG3, H.g3, H3, M, R, H3 * 2, (uint64_t)M * H3 * 2, 16, 1, 32, BF, NS) &&
         encode3d(&H.eG2, H.g2, H2, M, R, H2 * 2, (uint64_t)M * H2 * 2, 16, 1, 32, BF, NS) &&
         encode3d(&H.eG1, H.g1, (uint64_t)M * H1, 1, R, (uint64_t)M * H1 * 2, (uint64_t)M * H1 * 2, 16, 1, 32, BF, NS);
    if (!ok) {
      ctx->last_error = "cuTensorMapEncodeTiled failed for the activation maps";
      return FNN_E_CUDA;
    }
  }
  return FNN_OK;
}

fnn_status launch_aev_forward_bf16(fnn_ctx *ctx, const fnn_system *sys, const fnn_nlist *nl, __nv_bfloat16 *out,
                                   __nv_bfloat16 *out_lo, const int32_t *inv, cudaStream_t s);
fnn_status launch_aev_forward_fp8(fnn_ctx *ctx, const fnn_system *sys, const fnn_nlist *nl, uint8_t *out,
                                  float out_inv, const int32_t *inv, cudaStream_t s);
fnn_status launch_aev_l1_bf16(fnn_ctx *ctx, const fnn_system *sys, const fnn_nlist *nl, const CUtensorMap *mW1,
                              const float *b1cat, __nv_bfloat16 *h1, int M, cudaStream_t s);

static fnn_status f8_workspace(fnn_ctx *ctx, size_t rows) {
  TcState *t = state(ctx);
  F8 &f = t->f8;
  const int M = t->M;
  if (f.abuf && rows <= f.rows) return FNN_OK;
  ctx->gen++;
  rows = rows + rows / 8;
  if (f.abuf) cudaFree(f.abuf);
  f.abuf = nullptr;
  const size_t per_row = NAEV + (size_t)M * (H1 + H2 + H3 + H2 + H1);
  if (cudaMalloc(&f.abuf, rows * per_row) != cudaSuccess) {
    cudaGetLastError();
    ctx->last_error = "cudaMalloc failed for fp8 activations";
    return FNN_E_OOM;
  }
  f.rows = rows;
  const uint64_t R = rows;
  uint8_t *p = f.abuf;
  f.aev = p; p += rows * NAEV;
  f.h1 = p; p += rows * M * H1;
  f.h2 = p; p += rows * M * H2;
  f.g3 = p; p += rows * M * H3;
  f.g2 = p; p += rows * M * H2;
  f.g1 = p;
  const CUtensorMapDataType U8 = CU_TENSOR_MAP_DATA_TYPE_UINT8;
  bool ok = encode3d(&f.mAev, f.aev, NAEV, 1, R, NAEV, NAEV, 128, 1, 128, U8) &&
            encode3d(&f.mH1, f.h1, H1, M, R, H1, (uint64_t)M * H1, 128, 1, 128, U8) &&
            encode3d(&f.mH2, f.h2, H2, M, R, H2, (uint64_t)M * H2, 128, 1, 128, U8) &&
            encode3d(&f.mG3, f.g3, H3, M, R, H3, (uint64_t)M * H3, 128, 1, 128, U8) &&
            encode3d(&f.mG2, f.g2, H2, M, R, H2, (uint64_t)M * H2, 128, 1, 128, U8) &&
            encode3d(&f.mG1, f.g1, (uint64_t)M * H1, 1, R, (uint64_t)M * H1, (uint64_t)M * H1, 128, 1, 128, U8);
  const CUtensorMapSwizzle NS = CU_TENSOR_MAP_SWIZZLE_NONE;
  ok = ok && encode3d(&f.eH1, f.h1, H1, M, R, H1, (uint64_t)M * H1, 16, 1, 32, U8, NS) &&
       encode3d(&f.eH2, f.h2, H2, M, R, H2, (uint64_t)M * H2, 16, 1, 32, U8, NS) &&
       encode3d(&f.eG3, f.g3, H3, M, R, H3, (uint64_t)M * H3, 16, 1, 32, U8, NS) &&
       encode3d(&f.eG2, f.g2, H2, M, R, H2, (uint64_t)M * H2, 16, 1, 32, U8, NS) &&
       encode3d(&f.eG1, f.g1, (uint64_t)M * H1, 1, R, (uint64_t)M * H1, (uint64_t)M * H1, 16, 1, 32, U8, NS);
  if (!ok) {
    ctx->last_error = "cuTensorMapEncodeTiled failed for the fp8 activation maps";
    return FNN_E_CUDA;
  }
  return FNN_OK;
}

// max |x| over the rows of live tiles of a [rows][width] fp32 tensor, into *out (float bits)
__global__ void k_amax(const float *x, long long width, long long n, const int32_t *tile_elem, unsigned *out) {
  float mx = 0.f;
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x)
    if (tile_elem[k / width / ROW_TILE] >= 0) mx = fmaxf(mx, fabsf(x[k]));
  for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out, __float_as_uint(mx));
}

// Activation scales of the FP8 form from one FP32 evaluation of this system (synchronises the stream).
static fnn_status f8_calibrate(fnn_ctx *ctx, const fnn_system *sys, const fnn_nlist *nl, cudaStream_t s) {
  TcState *t = state(ctx);
  F8 &f = t->f8;
  fnn_status st;
  if ((st = ensure_workspace(ctx, nl->pad_cap))) return st;
  Workspace &ws = ctx->ws;
  if ((st = launch_aev_forward(ctx, sys, nl, ws.aev, nl->inv, s))) return st;
  if ((st = mlp_fp32_forward_backward(ctx, nl, s))) return st;
  if (!f.amax) FNN_CUDA_TRY(ctx, cudaMalloc(&f.amax, 6 * sizeof(unsigned)));
  FNN_CUDA_TRY(ctx, cudaMemsetAsync(f.amax, 0, 6 * sizeof(unsigned), s));
  const int M = t->M;
  const float *src[6] = {ws.aev, ws.h1, ws.h2, ws.g3, ws.g2, ws.g1};
  const long long width[6] = {NAEV, (long long)M * H1, (long long)M * H2, (long long)M * H3, (long long)M * H2,
                              (long long)M * H1};
  for (int k = 0; k < 6; k++) {
    FNN_KERNEL(ctx, "fp8_amax", s);
    k_amax<<<2 * ctx->num_sms, 256, 0, s>>>(src[k], width[k], (long long)nl->pad_cap * width[k], nl->tile_elem,
                                            f.amax + k);
  }
  if ((st = check_launch(ctx, "fp8_amax"))) return st;
  unsigned bits[6];
  FNN_CUDA_TRY(ctx, cudaMemcpyAsync(bits, f.amax, sizeof(bits), cudaMemcpyDeviceToHost, s));
  FNN_CUDA_TRY(ctx, cudaStreamSynchronize(s));
  for (int k = 0; k < 6; k++) {
    float a;
    memcpy(&a, &bits[k], sizeof a);
    f.act[k] = (a > 0.f && std::isfinite(a)) ? 2.f * a / 448.f : 1.f;
  }
  f.calibrated = true;
  return FNN_OK;
}

namespace {

// The six products (the third layer's two fused); the structure energies are reduced on the side
// stream as soon as the output layer is done, overlapping the backward products.
template <bool SPLIT>
fnn_status run_layers(fnn_ctx *ctx, TcState *t, const fnn_system *sys, const fnn_nlist *nl, double *E,
                      cudaStream_t s, bool l1_done = false) {
  constexpr int MODE = SPLIT ? tc::MODE_SPLIT : tc::MODE_BF16;
  const DeviceWeights &w = ctx->w;
  const Half &H = t->h[0], &L = t->h[SPLIT ? 1 : 0];
  const int M = w.M;
  const unsigned tiles = (unsigned)(nl->pad_cap / ROW_TILE);
  const char *nm[6] = {SPLIT ? "x3_l1_fwd" : "bf16_l1_fwd", SPLIT ? "x3_l2_fwd" : "bf16_l2_fwd",
                       nullptr, nullptr,
                       SPLIT ? "x3_l2_bwd" : "bf16_l2_bwd", SPLIT ? "x3_l1_bwd" : "bf16_l1_bwd"};
  fnn_status st;
  tc::Args a{};
  a.tile_elem = nl->tile_elem;
  a.st = ctx->status;
  a.M = M;
  // the partial last wave of the bias + CELU and CELU' products is cut into 64-column strips
  a.tail_nsplit = 1; a.nsub_w = 64; a.meta = nl->meta;
  // L1: all members at once, the n tile being the member; on two-SM tiles, each CTA of a pair staging its
  // rows and half of the member's weights (h1 is already there when the fused AEV kernel computed it)
  if (!l1_done) {
    const tc::PairArgs pa{NAEV, M, nl->meta, w.b1cat, (long long)M * H1, ctx->status};
    if ((st = launch_pair<MODE>(ctx, nm[0], &H.mAev, &L.mAev, &H.sW1, &L.sW1, &H.eH1, &L.eH1, pa, s))) return st;
  }
  // L2
  a.K = H1; a.N = H2; a.a_by_member = 1; a.b_by_member = 1;
  a.o_xm = 0; a.o_y = 1;
  a.bias = w.b2; a.bias_estride = H2; a.bias_mstride = (long long)NE * H2;
  {
    Maps m2{&H.mH1, &H.mW2, &L.mH1, &L.mW2, &H.eH2, &L.eH2, &H.eH2, &L.eH2};
    m2.Bs = &H.sW2; m2.Bs_lo = &L.sW2;
    if ((st = launch_q<192, tc::EPI_BIAS_CELU, MODE>(true, ctx, nm[1], m2, nullptr, a, dim3(1, tiles, M), s)))
      return st;
  }
  // L3 + output layer and the L3 backward g2 = (g3 W3) CELU'(h2) in one kernel (g3 stays in TMEM)
  {
    tc::L3Args l{};
    l.n_rowtiles = (int)tiles; l.n_members = M; l.tile_elem = nl->tile_elem;
    l.b3 = w.b3; l.w4 = w.w4; l.ypart = ctx->ws.ypart; l.M = M; l.scale = 1.f / (float)M; l.st = ctx->status;
    l.reverse = 1;   // the second-layer forward wrote the last tiles last
    // (64-byte operand rows: twice the ring stages for the same bytes in flight)
    const CUtensorMap *maps[10] = {&H.qH2, &L.qH2, &H.qW3, &L.qW3, &H.qW3T, &L.qW3T, &H.eH2, &L.eH2, &H.eG2, &L.eG2};
    if ((st = launch_l3_pair<MODE, 64>(ctx, SPLIT ? "x3_l3_pair" : "bf16_l3_pair", maps, l, s))) return st;
  }
  // side stream: the structure energies, and zeros for the tiles the first-layer input gradient's K parts
  // (the partial wave of its two-SM schedule on ncl1 clusters) are added into
  cudaLaunchConfig_t pcfg;
  cudaLaunchAttribute pattr[1];
  int ncl1;
  if ((st = pair_launch_config<MODE, tc::EPI_F32>(ctx, pcfg, pattr, ncl1, s))) return st;
  const int nt1 = (NAEV + 255) / 256, nkb1 = (M * H1 + 63) / 64;   // n tiles; K chunks of 64 elements
  if ((st = side_fork(ctx, s)) || (st = energy_reduce_rows(ctx, sys, nl, ctx->ws.ypart, 4, E, ctx->side)))
    return st;
  {
    FNN_KERNEL(ctx, "zero_tail", ctx->side);
    k_zero_tail_pair<<<ncl1 * 2 * ZT_PARTS, 64, 0, ctx->side>>>(nl->meta, nt1, ncl1, nkb1, NAEV, ctx->ws.gaev, NAEV);
  }
  // L2 backward: g1 = (g2 W2) CELU'(h1), stored member-concatenated for the L1 backward
  a.K = H2; a.N = H1; a.o_xm = H1; a.o_y = 0; a.x_y = 1;
  // (two aux buffers per warp keep its CELU' rows in flight; four-tile stages would leave room for one)
  {
    Maps m4{&H.mG2, &H.mW2T, &L.mG2, &L.mW2T, &H.eG1, &L.eG1, &H.eH1, &L.eH1};
    m4.Bs = &H.sW2T; m4.Bs_lo = &L.sW2T;
    if ((st = launch<256, tc::EPI_DCELU, MODE>(ctx, nm[4], m4, a, dim3(1, tiles, M), s))) return st;
  }
  a.tail_nsplit = 0;
  if ((st = side_join(ctx, s))) return st;
  // L1 backward on two-SM tiles: K = M*256 sums the members; fp32 dE/dAEV for the adjoint; the partial last
  // wave is split along K and added into the tiles zeroed above
  const CUtensorMap *og = gaev_map(ctx, t);
  if (!og) {
    ctx->last_error = "cuTensorMapEncodeTiled failed for the dE/dAEV map";
    return FNN_E_CUDA;
  }
  tc::PairArgs pb{M * H1, nt1, nl->meta, w.b1cat, 0, ctx->status};
  pb.N = NAEV;
  pb.tail_split = 1;
  {
    FNN_KERNEL(ctx, nm[5], s);
    FNN_CUDA_TRY(ctx, cudaLaunchKernelEx(&pcfg, tc::k_umma_pair<MODE, tc::EPI_F32>, H.mG1, L.mG1, H.sW1T, L.sW1T, *og,
                                         *og, pb));
  }
  return check_launch(ctx, nm[5]);
}

// The six products with e4m3 operands; scales as described at the top of this file.
fnn_status run_layers_f8(fnn_ctx *ctx, TcState *t, const fnn_nlist *nl, cudaStream_t s) {
  constexpr int MODE = tc::MODE_F8;
  const DeviceWeights &w = ctx->w;
  const F8 &f = t->f8;
  const int M = w.M;
  const long long MNE = (long long)M * NE;
  const unsigned tiles = (unsigned)(nl->pad_cap / ROW_TILE);
  fnn_status st;
  tc::Args a{};
  a.tile_elem = nl->tile_elem;
  a.st = ctx->status;
  a.M = M;
  // L1: member = n tile, on two-SM tiles (as the bf16 forms)
  {
    tc::PairArgs pa{NAEV, M, nl->meta, w.b1cat, (long long)M * H1, ctx->status};
    pa.a_scale = f.act[0]; pa.b_scale = f.wscale; pa.out_inv = 1.f / f.act[1];
    if ((st = launch_pair<MODE>(ctx, "fp8_l1_fwd", &f.mAev, &f.mAev, &f.sW1, &f.sW1, &f.eH1, &f.eH1, pa, s))) return st;
  }
  // L2
  a.K = H1; a.N = H2; a.a_by_member = 1; a.b_by_member = 1;
  a.o_xm = 0; a.o_y = 1;
  a.bias = w.b2; a.bias_estride = H2; a.bias_mstride = (long long)NE * H2;
  a.a_scale = f.act[1]; a.b_scale = f.wscale + 2 * MNE; a.b_scale_by = 1; a.out_inv = 1.f / f.act[2];
  if ((st = launch<192, tc::EPI_BIAS_CELU, MODE>(
           ctx, "fp8_l2_fwd", {&f.mH1, &f.mW2, &f.mH1, &f.mW2, &f.eH2, &f.eH2, &f.eH2, &f.eH2}, a,
           dim3(1, tiles, M), s)))
    return st;
  // L3 + output layer
  a.K = H2; a.N = H3;
  a.bias = w.b3; a.bias_estride = H3; a.bias_mstride = (long long)NE * H3;
  a.w4 = w.w4; a.w4_estride = H3; a.w4_mstride = (long long)NE * H3;
  a.ypart = ctx->ws.ypart; a.scale = 1.f / (float)M;
  a.a_scale = f.act[2]; a.b_scale = f.wscale + 4 * MNE; a.out_inv = 1.f / f.act[3];
  if ((st = launch<160, tc::EPI_L3, MODE>(
           ctx, "fp8_l3_fwd", {&f.mH2, &f.mW3, &f.mH2, &f.mW3, &f.eG3, &f.eG3, &f.eG3, &f.eG3}, a,
           dim3(1, tiles, M), s)))
    return st;
  // L3 backward
  a.K = H3; a.N = H2; a.x_y = 1;
  a.aux_scale = f.act[2];
  a.a_scale = f.act[3]; a.b_scale = f.wscale + 5 * MNE; a.out_inv = 1.f / f.act[4];
  if ((st = launch<192, tc::EPI_DCELU, MODE>(
           ctx, "fp8_l3_bwd", {&f.mG3, &f.mW3T, &f.mG3, &f.mW3T, &f.eG2, &f.eG2, &f.eH2, &f.eH2}, a,
           dim3(1, tiles, M), s)))
    return st;
  // L2 backward, stored member-concatenated
  a.K = H2; a.N = H1; a.o_xm = H1; a.o_y = 0;
  a.aux_scale = f.act[1];
  a.a_scale = f.act[4]; a.b_scale = f.wscale + 3 * MNE; a.out_inv = 1.f / f.act[5];
  if ((st = launch<256, tc::EPI_DCELU, MODE>(
           ctx, "fp8_l2_bwd", {&f.mG2, &f.mW2T, &f.mG2, &f.mW2T, &f.eG1, &f.eG1, &f.eH1, &f.eH1}, a,
           dim3(1, tiles, M), s)))
    return st;
  // L1 backward: K = M*256 sums the members (one W1^T scale per element); fp32 dE/dAEV
  a.K = M * H1; a.N = NAEV; a.a_by_member = 0; a.b_by_member = 0;
  a.out = ctx->ws.gaev; a.ldo = NAEV; a.o_mstride = 0; a.scale = 1.f;
  a.a_scale = f.act[5]; a.b_scale = f.wscale + 1 * MNE; a.b_scale_by = 0;
  const CUtensorMap *og = gaev_map(ctx, t);
  if (!og) {
    ctx->last_error = "cuTensorMapEncodeTiled failed for the dE/dAEV map";
    return FNN_E_CUDA;
  }
  return launch<256, tc::EPI_F32, MODE>(ctx, "fp8_l1_bwd", {&f.mG1, &f.mW1T, &f.mG1, &f.mW1T, og, og, &f.mG1, &f.mG1},
                                        a, dim3((NAEV + 255) / 256, tiles, 1), s);
}

}  // namespace

fnn_status fp8_calibrate(fnn_ctx *ctx, const fnn_system *sys, const fnn_nlist *nl, cudaStream_t s) {
  TcState *t = state(ctx);
  if (!t->f8.wbuf || t->M != ctx->w.M) {
    ctx->last_error = "fp8 weights missing";
    return FNN_E_STATE;
  }
  return f8_calibrate(ctx, sys, nl, s);
}

// AEV (bf16, or hi/lo pairs) -> six tcgen05 GEMMs -> member-averaged energies; dE/dAEV (fp32) in ws.gaev.
// FNN_BF16_FUSED computes the AEV and the first product in one kernel (aev.cu, k_aev_l1).
fnn_status tc_energy(fnn_ctx *ctx, const fnn_system *sys, const fnn_nlist *nl, fnn_precision prec, double *E,
                     cudaStream_t s) {
  const bool split = prec == FNN_FP32X3;
  TcState *t = state(ctx);
  if (!t->wbuf || t->M != ctx->w.M) {
    ctx->last_error = "bf16 weights missing";
    return FNN_E_STATE;
  }
  fnn_status st;
  if (prec == FNN_FP8) {
    if (!t->f8.calibrated && (st = f8_calibrate(ctx, sys, nl, s))) return st;
    if ((st = f8_workspace(ctx, nl->pad_cap))) return st;
    if ((st = launch_aev_forward_fp8(ctx, sys, nl, t->f8.aev, 1.f / t->f8.act[0], nl->inv, s))) return st;
    if ((st = run_layers_f8(ctx, t, nl, s))) return st;
    return energy_reduce_rows(ctx, sys, nl, ctx->ws.ypart, 4, E, s);
  }
  if ((st = tc_workspace(ctx, nl->pad_cap, split ? 2 : 1))) return st;
  if (prec == FNN_BF16_FUSED) {   // AEV and first layer in one kernel, then the other five products
    if ((st = launch_aev_l1_bf16(ctx, sys, nl, &t->h[0].mW1, ctx->w.b1cat, t->h[0].h1, t->M, s))) return st;
    return run_layers<false>(ctx, t, sys, nl, E, s, true);
  }
  if ((st = launch_aev_forward_bf16(ctx, sys, nl, t->h[0].aev, split ? t->h[1].aev : nullptr, nl->inv, s))) return st;
  return split ? run_layers<true>(ctx, t, sys, nl, E, s) : run_layers<false>(ctx, t, sys, nl, E, s);
}


// ============================================================================================ training
// Parameter gradients of the loss with BF16 networks on the tensor cores (the FP32 form of this
// computation, with the derivation, is in train.cu).  Activations and gradient streams are bf16 in
// HBM; every product accumulates in FP32:
//   forward   h_l = CELU(h_{l-1} W_l^T + b_l)                           (EPI_BIAS_CELU)
//   tangent   hd_l = CELU'(h_l) (hd_{l-1} W_l^T), hd_0 = J dL/dF         (EPI_DCELU, aux h_l)
//   reverse   raw gb_{l-1} = gbz_l W_l, g_{l-1} = gz_l W_l               (EPI_PLAIN)
//             gbz = CELU'(h) gb, gz = CELU'(h) g + (CELU''/CELU')(h) hd gb   (k_act_reverse_bf16)
//   weights   dW_l += gbz_l^T hd_{l-1} + gz_l^T h_{l-1}: K runs over each element's rows; both factors are
//             read in place as MN-major operands (64 rows x 64 features per box) (MODE_WG, EPI_ATOMIC)

namespace {

__device__ __forceinline__ float dcelu_hb(float h) { return h > 0.f ? 1.f : 1.f + h * CELU_INV_ALPHA; }
__device__ __forceinline__ float ratio_hb(float h) { return h > 0.f ? 0.f : CELU_INV_ALPHA; }

// output layer: gbz3 = CELU'(h3) (-(1/M) w4), gz3 = CELU'(h3) ((1/M) dL/dE w4) + ratio(h3) hd3 gb3;
// dw4 += (1/M) dL/dE h3 - (1/M) hd3, db4 += (1/M) dL/dE, db3 += gz3 (sums per tile, one atomic each).
// blockDim = H3: thread (feature group fg of 8, row lane rl of 8) moves 16 bytes per array and row
__global__ void __launch_bounds__(H3) k_out_reverse_bf16(int M, const int32_t *tile_elem, const int32_t *inv,
                                                         const int32_t *atom_mol, const double *dLdE, const float *w4,
                                                         const __nv_bfloat16 *h3, const __nv_bfloat16 *hd3,
                                                         __nv_bfloat16 *gbz3, __nv_bfloat16 *gz3, float *dw4,
                                                         float *db4, float *db3) {
  __shared__ float red_w[8][H3], red_b3[8][H3];
  __shared__ float red_b[8];
  constexpr int G8 = H3 / 8;
  const int tile = blockIdx.x, m = blockIdx.y;
  const int e = tile_elem[tile];
  if (e < 0) return;
  const int fg = threadIdx.x % G8, rl = threadIdx.x / G8;
  const float c = 1.f / (float)M;
  float w[8];
#pragma unroll
  for (int j = 0; j < 8; j++) w[j] = w4[((size_t)m * NE + e) * H3 + 8 * fg + j];
  float acc_w[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f}, acc_b3[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  float acc_b = 0.f;
  for (int rr = rl; rr < ROW_TILE; rr += 8) {
    const size_t r = (size_t)tile * ROW_TILE + rr;
    const int i = inv[r];
    const size_t o = r * (size_t)M * H3 + (size_t)m * H3 + 8 * fg;
    const int mol = i < 0 ? -1 : atom_mol[i];
    alignas(16) __nv_bfloat16 hv[8], hdv[8], ob[8], oz[8];
    if (mol < 0) {
      *reinterpret_cast<uint4 *>(gbz3 + o) = make_uint4(0u, 0u, 0u, 0u);
      *reinterpret_cast<uint4 *>(gz3 + o) = make_uint4(0u, 0u, 0u, 0u);
      continue;
    }
    const float cE = (float)dLdE[mol] * c;
    *reinterpret_cast<uint4 *>(hv) = *reinterpret_cast<const uint4 *>(h3 + o);
    *reinterpret_cast<uint4 *>(hdv) = *reinterpret_cast<const uint4 *>(hd3 + o);
#pragma unroll
    for (int j = 0; j < 8; j++) {
      const float h = __bfloat162float(hv[j]), hd = __bfloat162float(hdv[j]);
      const float s1 = dcelu_hb(h);
      const float gb = -c * w[j], g = cE * w[j];
      const float gz = s1 * g + ratio_hb(h) * hd * gb;
      ob[j] = __float2bfloat16(s1 * gb);
      oz[j] = __float2bfloat16(gz);
      acc_w[j] += cE * h - c * hd;
      acc_b3[j] += gz;
    }
    *reinterpret_cast<uint4 *>(gbz3 + o) = *reinterpret_cast<const uint4 *>(ob);
    *reinterpret_cast<uint4 *>(gz3 + o) = *reinterpret_cast<const uint4 *>(oz);
    acc_b += cE;
  }
#pragma unroll
  for (int j = 0; j < 8; j++) {
    red_w[rl][8 * fg + j] = acc_w[j];
    red_b3[rl][8 * fg + j] = acc_b3[j];
  }
  if (fg == 0) red_b[rl] = acc_b;
  __syncthreads();
  const int n = threadIdx.x;
  float tw = 0.f, tb3 = 0.f;
#pragma unroll
  for (int q = 0; q < 8; q++) {
    tw += red_w[q][n];
    tb3 += red_b3[q][n];
  }
  atomicAdd(&dw4[((size_t)m * NE + e) * H3 + n], tw);
  atomicAdd(&db3[((size_t)m * NE + e) * H3 + n], tb3);
  if (n == 0) {
    float tb = 0.f;
#pragma unroll
    for (int q = 0; q < 8; q++) tb += red_b[q];
    atomicAdd(&db4[(size_t)m * NE + e], tb);
  }
}

// hidden layer: (raw gb, g) -> gbz = CELU'(h) gb, gz = CELU'(h) g + ratio(h) hd gb; db += gz per tile.
// blockDim = F: thread (feature group fg of 8, row lane rl of 8) moves 16 bytes per array and row
__global__ void __launch_bounds__(256) k_act_reverse_bf16(int M, int F, const int32_t *tile_elem,
                                                          const __nv_bfloat16 *h, const __nv_bfloat16 *hd,
                                                          const __nv_bfloat16 *gb, const __nv_bfloat16 *g,
                                                          __nv_bfloat16 *gbz, __nv_bfloat16 *gz, float *db) {
  __shared__ float red[8][256];
  const int tile = blockIdx.x, m = blockIdx.y;
  const int e = tile_elem[tile];
  if (e < 0) return;
  const int G8 = F / 8, fg = threadIdx.x % G8, rl = threadIdx.x / G8;
  float acc[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  for (int rr = rl; rr < ROW_TILE; rr += 8) {
    const size_t o = ((size_t)tile * ROW_TILE + rr) * (size_t)M * F + (size_t)m * F + 8 * fg;
    alignas(16) __nv_bfloat16 hv[8], hdv[8], gbv[8], gv[8], ob[8], oz[8];
    *reinterpret_cast<uint4 *>(hv) = *reinterpret_cast<const uint4 *>(h + o);
    *reinterpret_cast<uint4 *>(hdv) = *reinterpret_cast<const uint4 *>(hd + o);
    *reinterpret_cast<uint4 *>(gbv) = *reinterpret_cast<const uint4 *>(gb + o);
    *reinterpret_cast<uint4 *>(gv) = *reinterpret_cast<const uint4 *>(g + o);
#pragma unroll
    for (int j = 0; j < 8; j++) {
      const float x = __bfloat162float(hv[j]), b = __bfloat162float(gbv[j]);
      const float s1 = dcelu_hb(x);
      const float z = s1 * __bfloat162float(gv[j]) + ratio_hb(x) * __bfloat162float(hdv[j]) * b;
      ob[j] = __float2bfloat16(s1 * b);
      oz[j] = __float2bfloat16(z);
      acc[j] += z;
    }
    *reinterpret_cast<uint4 *>(gbz + o) = *reinterpret_cast<const uint4 *>(ob);
    *reinterpret_cast<uint4 *>(gz + o) = *reinterpret_cast<const uint4 *>(oz);
  }
#pragma unroll
  for (int j = 0; j < 8; j++) red[rl][8 * fg + j] = acc[j];
  __syncthreads();
  if ((int)threadIdx.x < F) {
    float t = 0.f;
#pragma unroll
    for (int r = 0; r < 8; r++) t += red[r][threadIdx.x];
    atomicAdd(&db[((size_t)m * NE + e) * F + threadIdx.x], t);
  }
}

struct TrainTc {
  size_t rows = 0;
  int M = 0;
  void *buf = nullptr;
  __nv_bfloat16 *t = nullptr, *h3 = nullptr, *hd1 = nullptr, *hd2 = nullptr, *hd3 = nullptr;   // t: AEV tangent
  __nv_bfloat16 *gbz3 = nullptr, *gz3 = nullptr, *gb2 = nullptr, *g2 = nullptr, *gbz2 = nullptr, *gz2 = nullptr;
  __nv_bfloat16 *gb1 = nullptr, *g1 = nullptr, *gbz1 = nullptr, *gz1 = nullptr;
  // operand maps (128-byte rows), epilogue piece maps, MN-major weight-gradient operand maps
  CUtensorMap mT, mHD1, mHD2, mGBZ3, mGZ3, mGBZ2, mGZ2;
  CUtensorMap eH3, eHD1, eHD2, eHD3, eGB2, eG2, eGB1, eG1;
  CUtensorMap wGBZ3, wGZ3, wGBZ2, wGZ2, wGBZ1, wGZ1, wHD2, wHD1, wT;
};

}  // namespace

void free_train_tc(void *p) {
  TrainTc *T = static_cast<TrainTc *>(p);
  if (!T) return;
  if (T->buf) cudaFree(T->buf);
  delete T;
}

static fnn_status train_tc_workspace(fnn_ctx *ctx, TcState *ts, size_t rows) {
  if (!ts->train) ts->train = new TrainTc();
  TrainTc &T = *static_cast<TrainTc *>(ts->train);
  const int M = ts->M;
  if (T.buf && rows <= T.rows && T.M == M) return FNN_OK;
  if (T.buf) cudaFree(T.buf);
  T.buf = nullptr;
  rows = (rows + rows / 8 + 127) / 128 * 128;
  const size_t R = rows;
  const size_t n16 = R * (NAEV + (size_t)M * (H3 + H1 + H2 + H3 + 2 * H3 + 4 * H2 + 4 * H1));
  const size_t bytes = n16 * sizeof(__nv_bfloat16) + 4096;
  if (cudaMalloc(&T.buf, bytes) != cudaSuccess) {
    cudaGetLastError();
    ctx->last_error = "cudaMalloc failed for the bf16 training workspace";
    return FNN_E_OOM;
  }
  __nv_bfloat16 *p = static_cast<__nv_bfloat16 *>(T.buf);
  auto take = [&](size_t n) {
    __nv_bfloat16 *q = p;
    p += n;
    return q;
  };
  T.t = take(R * NAEV);
  T.h3 = take(R * M * H3);
  T.hd1 = take(R * M * H1);
  T.hd2 = take(R * M * H2);
  T.hd3 = take(R * M * H3);
  T.gbz3 = take(R * M * H3);
  T.gz3 = take(R * M * H3);
  T.gb2 = take(R * M * H2);
  T.g2 = take(R * M * H2);
  T.gbz2 = take(R * M * H2);
  T.gz2 = take(R * M * H2);
  T.gb1 = take(R * M * H1);
  T.g1 = take(R * M * H1);
  T.gbz1 = take(R * M * H1);
  T.gz1 = take(R * M * H1);
  const CUtensorMapDataType BF = CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
  const CUtensorMapSwizzle NS = CU_TENSOR_MAP_SWIZZLE_NONE, S128 = CU_TENSOR_MAP_SWIZZLE_128B;
  auto op = [&](CUtensorMap *mp, void *b, uint64_t F) {   // row-major operand, member in the middle
    return encode3d(mp, b, F, M, R, F * 2, (uint64_t)M * F * 2, 64, 1, 128, BF, S128);
  };
  auto ep = [&](CUtensorMap *mp, void *b, uint64_t F) {   // epilogue pieces
    return encode3d(mp, b, F, M, R, F * 2, (uint64_t)M * F * 2, 16, 1, 32, BF, NS);
  };
  auto wn = [&](CUtensorMap *mp, void *b, uint64_t F) {   // MN-major boxes: 64 features x 64 rows
    return encode3d(mp, b, F, M, R, F * 2, (uint64_t)M * F * 2, 64, 1, 64, BF, S128);
  };
  bool ok = encode3d(&T.mT, T.t, NAEV, 1, R, NAEV * 2, NAEV * 2, 64, 1, 128, BF, S128) && op(&T.mHD1, T.hd1, H1) &&
            op(&T.mHD2, T.hd2, H2) && op(&T.mGBZ3, T.gbz3, H3) && op(&T.mGZ3, T.gz3, H3) && op(&T.mGBZ2, T.gbz2, H2) &&
            op(&T.mGZ2, T.gz2, H2) && ep(&T.eH3, T.h3, H3) && ep(&T.eHD1, T.hd1, H1) && ep(&T.eHD2, T.hd2, H2) &&
            ep(&T.eHD3, T.hd3, H3) && ep(&T.eGB2, T.gb2, H2) && ep(&T.eG2, T.g2, H2) && ep(&T.eGB1, T.gb1, H1) &&
            ep(&T.eG1, T.g1, H1) && wn(&T.wGBZ3, T.gbz3, H3) && wn(&T.wGZ3, T.gz3, H3) && wn(&T.wGBZ2, T.gbz2, H2) &&
            wn(&T.wGZ2, T.gz2, H2) && wn(&T.wGBZ1, T.gbz1, H1) && wn(&T.wGZ1, T.gz1, H1) && wn(&T.wHD2, T.hd2, H2) &&
            wn(&T.wHD1, T.hd1, H1) && encode3d(&T.wT, T.t, NAEV, 1, R, NAEV * 2, NAEV * 2, 64, 1, 64, BF, S128);
  if (!ok) {
    ctx->last_error = "cuTensorMapEncodeTiled failed for the training maps";
    return FNN_E_CUDA;
  }
  T.rows = rows;
  T.M = M;
  return FNN_OK;
}

fnn_status tc_param_grads(fnn_ctx *ctx, const fnn_system *sys, const fnn_nlist *nl, const double *dLdE,
                          const float *dLdF, const fnn_grads *g, cudaStream_t s) {
  TcState *ts = state(ctx);
  if (!ts->wbuf || ts->M != ctx->w.M) {
    ctx->last_error = "bf16 weights missing";
    return FNN_E_STATE;
  }
  fnn_status st;
  if ((st = ensure_workspace(ctx, nl->pad_cap)) || (st = tc_workspace(ctx, nl->pad_cap, 1)) ||
      (st = train_tc_workspace(ctx, ts, nl->pad_cap)))
    return st;
  TrainTc &T = *static_cast<TrainTc *>(ts->train);
  const Half &H = ts->h[0];
  const DeviceWeights &w = ctx->w;
  const int M = w.M;
  const int rows = nl->pad_cap;
  const unsigned tiles = (unsigned)(rows / ROW_TILE);
  constexpr int B16 = tc::MODE_BF16;
  // AEV and its tangent along dL/dF (bf16), in one pass over the triplets
  if ((st = launch_aev_tangent_bf16(ctx, sys, nl, dLdF, T.t, H.aev, nl->inv, s))) return st;
  tc::Args a{};
  a.tile_elem = nl->tile_elem;
  a.st = ctx->status;
  a.M = M;
  // ---- forward h1, h2, h3
  {   // (two-SM tiles, as in the forward step)
    const tc::PairArgs pa{NAEV, M, nl->meta, w.b1cat, (long long)M * H1, ctx->status};
    if ((st = launch_pair<B16>(ctx, "tr16_l1_fwd", &H.mAev, &H.mAev, &H.sW1, &H.sW1, &H.eH1, &H.eH1, pa, s))) return st;
  }
  a.K = H1; a.N = H2; a.a_by_member = 1; a.b_by_member = 1; a.o_y = 1;
  a.bias = w.b2; a.bias_estride = H2; a.bias_mstride = (long long)NE * H2;
  if ((st = launch<192, tc::EPI_BIAS_CELU, B16>(ctx, "tr16_l2_fwd",
                                                {&H.mH1, &H.mW2, &H.mH1, &H.mW2, &H.eH2, &H.eH2, &H.eH2, &H.eH2}, a,
                                                dim3(1, tiles, M), s)))
    return st;
  a.K = H2; a.N = H3;
  a.bias = w.b3; a.bias_estride = H3; a.bias_mstride = (long long)NE * H3;
  if ((st = launch<160, tc::EPI_BIAS_CELU, B16>(ctx, "tr16_l3_fwd",
                                                {&H.mH2, &H.mW3, &H.mH2, &H.mW3, &T.eH3, &T.eH3, &T.eH3, &T.eH3}, a,
                                                dim3(1, tiles, M), s)))
    return st;
  // ---- tangents hd1, hd2, hd3
  a.K = NAEV; a.N = M * H1; a.a_by_member = 0; a.b_by_member = 0; a.o_y = 2; a.x_y = 2;
  if ((st = launch<256, tc::EPI_DCELU, B16>(ctx, "tr16_l1_tan",
                                            {&T.mT, &H.mW1, &T.mT, &H.mW1, &T.eHD1, &T.eHD1, &H.eH1, &H.eH1}, a,
                                            dim3(M, tiles, 1), s)))
    return st;
  a.K = H1; a.N = H2; a.a_by_member = 1; a.b_by_member = 1; a.o_y = 1; a.x_y = 1;
  if ((st = launch<192, tc::EPI_DCELU, B16>(ctx, "tr16_l2_tan",
                                            {&T.mHD1, &H.mW2, &T.mHD1, &H.mW2, &T.eHD2, &T.eHD2, &H.eH2, &H.eH2}, a,
                                            dim3(1, tiles, M), s)))
    return st;
  a.K = H2; a.N = H3;
  if ((st = launch<160, tc::EPI_DCELU, B16>(ctx, "tr16_l3_tan",
                                            {&T.mHD2, &H.mW3, &T.mHD2, &H.mW3, &T.eHD3, &T.eHD3, &T.eH3, &T.eH3}, a,
                                            dim3(1, tiles, M), s)))
    return st;
  // ---- output layer reverse (+ dw4, db4, db3)
  {
    FNN_KERNEL(ctx, "tr16_out_rev", s);
    k_out_reverse_bf16<<<dim3(tiles, M), H3, 0, s>>>(M, nl->tile_elem, nl->inv, nl->atom_mol, dLdE, w.w4, T.h3,
                                                      T.hd3, T.gbz3, T.gz3, g->w4, g->b4, g->b3);
  }
  // ---- layer 3 reverse: raw gb2 = gbz3 W3, g2 = gz3 W3, then the activation reverse at layer 2
  a.K = H3; a.N = H2; a.a_by_member = 1; a.b_by_member = 1; a.o_y = 1;
  if ((st = launch<192, tc::EPI_PLAIN, B16>(ctx, "tr16_l3_rev",
                                            {&T.mGBZ3, &H.mW3T, &T.mGBZ3, &H.mW3T, &T.eGB2, &T.eGB2, &T.eGB2, &T.eGB2},
                                            a, dim3(1, tiles, M), s)))
    return st;
  if ((st = launch<192, tc::EPI_PLAIN, B16>(ctx, "tr16_l3_rev",
                                            {&T.mGZ3, &H.mW3T, &T.mGZ3, &H.mW3T, &T.eG2, &T.eG2, &T.eG2, &T.eG2}, a,
                                            dim3(1, tiles, M), s)))
    return st;
  {
    FNN_KERNEL(ctx, "tr16_act_rev", s);
    k_act_reverse_bf16<<<dim3(tiles, M), H2, 0, s>>>(M, H2, nl->tile_elem, H.h2, T.hd2, T.gb2, T.g2, T.gbz2, T.gz2,
                                                      g->b2);
  }
  // ---- layer 2 reverse
  a.K = H2; a.N = H1;
  if ((st = launch<256, tc::EPI_PLAIN, B16>(ctx, "tr16_l2_rev",
                                            {&T.mGBZ2, &H.mW2T, &T.mGBZ2, &H.mW2T, &T.eGB1, &T.eGB1, &T.eGB1, &T.eGB1},
                                            a, dim3(1, tiles, M), s)))
    return st;
  if ((st = launch<256, tc::EPI_PLAIN, B16>(ctx, "tr16_l2_rev",
                                            {&T.mGZ2, &H.mW2T, &T.mGZ2, &H.mW2T, &T.eG1, &T.eG1, &T.eG1, &T.eG1}, a,
                                            dim3(1, tiles, M), s)))
    return st;
  {
    FNN_KERNEL(ctx, "tr16_act_rev", s);
    k_act_reverse_bf16<<<dim3(tiles, M), H1, 0, s>>>(M, H1, nl->tile_elem, H.h1, T.hd1, T.gb1, T.g1, T.gbz1, T.gz1,
                                                      g->b1);
  }
  // ---- weight gradients: dW_l += gbz_l^T hd_{l-1} + gz_l^T h_{l-1} over each element's rows
  tc::Args wg{};
  wg.st = ctx->status;
  wg.M = M;
  wg.seg = nl->meta + META_SEG;
  wg.kchunk = 1024;   // rows per work item: about four waves on 148 SMs for the 148,565-row batch (4096: two)
  wg.n_chunks = (rows + wg.kchunk - 1) / wg.kchunk;
  constexpr int WG = tc::MODE_WG;
  wg.K = 0;
  // dW[m][e] (O x I, fp32) as the reduce-add target of each product: boxes of 32 rows x 8 columns
  CUtensorMap d3, d2, d1;
  auto dmap = [&](CUtensorMap *mp, float *dW, uint64_t O, uint64_t I) {
    return encode3d(mp, dW, I, O, (uint64_t)M * NE, I * 4, O * I * 4, 8, 32, 1, CU_TENSOR_MAP_DATA_TYPE_FLOAT32,
                    CU_TENSOR_MAP_SWIZZLE_NONE);
  };
  if (!dmap(&d3, g->W3, H3, H2) || !dmap(&d2, g->W2, H2, H1) || !dmap(&d1, g->W1, H1, NAEV)) {
    ctx->last_error = "cuTensorMapEncodeTiled failed for the weight-gradient maps";
    return FNN_E_CUDA;
  }
  wg.N = H2; wg.O = H3;
  if ((st = launch<192, tc::EPI_ATOMIC, WG>(ctx, "tr16_l3_wgrad", {&T.wGBZ3, &T.wHD2, &T.wGZ3, &H.wH2, &d3, &d3, &d3, &d3},
                                            wg, dim3(1, (H3 + 127) / 128, wg.n_chunks * M * NE), s)))
    return st;
  wg.N = H1; wg.O = H2;
  if ((st = launch<256, tc::EPI_ATOMIC, WG>(ctx, "tr16_l2_wgrad", {&T.wGBZ2, &T.wHD1, &T.wGZ2, &H.wH1, &d2, &d2, &d2, &d2},
                                            wg, dim3(1, (H2 + 127) / 128, wg.n_chunks * M * NE), s)))
    return st;
  wg.N = NAEV; wg.O = H1; wg.b_shared = 1;
  return launch<256, tc::EPI_ATOMIC, WG>(ctx, "tr16_l1_wgrad", {&T.wGBZ1, &T.wT, &T.wGZ1, &H.wAev, &d1, &d1, &d1, &d1},
                                         wg, dim3((NAEV + 255) / 256, (H1 + 127) / 128, wg.n_chunks * M * NE), s);
}

}  // namespace fnn
