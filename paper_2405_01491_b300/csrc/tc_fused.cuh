// Fused third layer, forward and backward, of the per-element networks on the tensor cores (the
// bf16 and three-term split forms).  For a 128-row tile of one element and member:
//   G1  z3 = h2 W3^T                       K = 192, N = 160; accumulator in TMEM region Z[k & 1]
//   E1  y += CELU(z3 + b3) . w4 (row partial sums) and g3 = (1/M) w4 CELU'(z3 + b3), written back
//       into the same TMEM columns as packed bf16: the 16 columns c .. c+15 of a piece become the
//       hi halves of g3[c .. c+15] (columns c .. c+7, two per column) and the lo halves (c+8 .. c+15)
//   G2  g3 W3                              K = 160, N = 192; A read from TMEM (16 K elements per
//       instruction: hi at column 16 j, lo at 16 j + 8), accumulator in TMEM region G
//   E2  g2 = (g3 W3) CELU'(h2), with h2 (the aux rows) loaded by TMA, stored by TMA (hi, lo)
// so g3 never leaves the SM and h2 is read for both products in one pass over the tiles (the
// unfused form writes and re-reads g3 and reads h2 twice).  Section II.B defines the networks; the
// backward product is the chain rule through their third layer.
//
// TMEM: Z0 = columns [0, 160), Z1 = [160, 320), G = [320, 512).  The MMA thread issues, for the k-th
// tile of this CTA, G1(k) and then G2(k - 1), so E1(k) runs while G2(k - 1) is on the tensor pipe
// and E2(k - 1) while G1(k + 1) is.  Every wait is bounded as in tc_gemm.cuh.
#pragma once

#include "tc_gemm.cuh"

namespace fnn {
namespace tc {

// D[tmem] (+)= A[tmem] * B[smem]^T, bf16 inputs, fp32 accumulation (A: lane = row, 2 K elements per column)
__device__ __forceinline__ void mma_bf16_ts(uint32_t d, uint32_t a_tmem, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n\t}\n" ::"r"(d),
      "r"(a_tmem), "l"(b), "r"(idesc), "r"(acc));
}

// 32 TMEM lanes x 16 consecutive 32-bit columns from thread t's r[0..15] into lane (base + t)
__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t r[16]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};" ::"r"(
          taddr),
      "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]), "r"(r[8]), "r"(r[9]),
      "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15])
      : "memory");
}
__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// 2^x on the special-function unit (ex2.approx.ftz, arguments <= 0 here); exp(x) = 2^(x log2 e)
constexpr float LOG2E = 1.4426950408889634f;
__device__ __forceinline__ float exp2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

struct L3Args {
  int n_rowtiles, n_members;
  const int32_t *tile_elem;    // element of each 128-row tile (-1: skip)
  const float *b3, *w4;        // [M][7][160]
  float *ypart;                // [rows][M][4]: column `part` of each epilogue warp quarter
  int M;
  float scale;                 // 1/M
  DevStatus *st;
  int reverse;                 // tiles last to first: h2's most recently written tiles (still in L2) first
};

constexpr int L3_N1 = H3, L3_N2 = H2, L3_K1 = H2, L3_K2 = H3;
constexpr int L3_ZCOLS = 160, L3_GCOL = 320;
constexpr int L3_PIECES = 3;   // E2 pieces per epilogue warp: columns 16 part + {0, 64, 128} of 192

template <int MODE, int KB>
struct L3Smem {
  static constexpr bool SPLIT = MODE == MODE_SPLIT;
  static constexpr int OB = SPLIT ? 2 : 1;      // halves per output buffer
  static constexpr int WBUF = 1024;             // 32 rows x 16 bf16
  // aux / output buffers per epilogue warp: one per E2 piece, two for the split (whose stages are larger)
  static constexpr int NAUX = SPLIT ? 2 : L3_PIECES;
  static constexpr int OBYTES = EPI_WARPS * NAUX * OB * WBUF;
  static constexpr int BROWS = L3_N2 > L3_N1 ? L3_N2 : L3_N1;
  static constexpr int FIXED = OBYTES + 2048;
  // a split stage holds hi and lo of both operands for one K chunk (three products per K step)
  static constexpr int FIT = (SMEM_LIMIT - FIXED) / (OB * (BM * KB + BROWS * KB));
  static constexpr int CAP = 6 * (BKB / KB);
  static constexpr int STAGES = FIT > CAP ? CAP : FIT;
  uint8_t A[STAGES][OB * BM * KB];
  uint8_t B[STAGES][OB * BROWS * KB];
  uint8_t O[OBYTES];
  uint64_t full[STAGES], empty[STAGES];
  uint64_t z_full[2], a_full[2], g_full, g_empty, fin, aux_bar[EPI_WARPS][NAUX];
  uint32_t tmem_base;
  int abort_flag;
};

template <int MODE, int KB>
constexpr size_t l3_smem_bytes() {
  return sizeof(L3Smem<MODE, KB>) + 1024;
}

// tile t -> (row tile, member, element); false for padding tiles
__device__ __forceinline__ bool l3_tile(const L3Args &p, int t, int &rt, int &m, int &e) {
  if (p.reverse) t = p.n_rowtiles * p.n_members - 1 - t;
  rt = t % p.n_rowtiles;
  m = t / p.n_rowtiles;
  e = p.tile_elem[rt];
  return e >= 0;
}

template <int MODE, int KB>
__global__ void __launch_bounds__(THREADS, 1)
    k_l3_pair(const __grid_constant__ CUtensorMap tmH2, const __grid_constant__ CUtensorMap tmH2_lo,
              const __grid_constant__ CUtensorMap tmW3, const __grid_constant__ CUtensorMap tmW3_lo,
              const __grid_constant__ CUtensorMap tmW3T, const __grid_constant__ CUtensorMap tmW3T_lo,
              const __grid_constant__ CUtensorMap tmX, const __grid_constant__ CUtensorMap tmX_lo,
              const __grid_constant__ CUtensorMap tmO, const __grid_constant__ CUtensorMap tmO_lo, L3Args p) {
  static_assert(MODE == MODE_SPLIT || MODE == MODE_BF16, "bf16 operands");
  static_assert(KB == 128 || KB == 64, "operand row width");
  using SM = L3Smem<MODE, KB>;
  static_assert(SM::STAGES >= 2 && sizeof(SM) + 1024 <= SMEM_LIMIT, "shared memory budget");
  constexpr bool SPLIT = MODE == MODE_SPLIT;
  constexpr int STAGES = SM::STAGES;
  constexpr int BK = KB / 2;                               // bf16 K elements per stage
  constexpr int NK1 = (L3_K1 + BK - 1) / BK, NK2 = (L3_K2 + BK - 1) / BK;   // 3, 3 (128-byte rows) or 6, 5
  extern __shared__ uint8_t smem_raw[];
  SM &S = *reinterpret_cast<SM *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int T = p.n_rowtiles * p.n_members;
  volatile int *abort_flag = &S.abort_flag;

  if (warp == 0 && lane == 0) {
    for (int s = 0; s < STAGES; s++) {
      mbar_init(&S.full[s], 1);
      mbar_init(&S.empty[s], 1);
    }
    for (int a = 0; a < 2; a++) {
      mbar_init(&S.z_full[a], 1);
      mbar_init(&S.a_full[a], EPI_WARPS);
    }
    for (int w = 0; w < EPI_WARPS; w++)
      for (int b = 0; b < SM::NAUX; b++) mbar_init(&S.aux_bar[w][b], 1);
    mbar_init(&S.g_full, 1);
    mbar_init(&S.g_empty, EPI_WARPS);
    mbar_init(&S.fin, 1);
    S.abort_flag = 0;
    fence_barrier_init();
  }
  if (warp == 1) {
    tmem_alloc(&S.tmem_base, 2 * TMEM_COLS);
    tmem_relinquish();
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = S.tmem_base;

  if (warp == 0) {
    if (lane == 0) {  // ---- TMA producer, in the MMA thread's order: G1(0), then G1(k), G2(k - 1)
      long long g = 0, issued = 0;
      int prev = -1;   // previous valid tile of this CTA (its G2 is still to load)
      for (int t = blockIdx.x;; t += gridDim.x) {
        int rt = 0, m = 0, e = 0;
        const bool have = t < T;
        if (have && !l3_tile(p, t, rt, m, e)) continue;
        if (*abort_flag) break;
        for (int phase = 0; phase < 2; phase++) {
          int trt, tm, te;
          if (phase == 0) {
            if (!have) continue;
            trt = rt; tm = m; te = e;
          } else {
            if (prev < 0) continue;
            l3_tile(p, prev, trt, tm, te);
          }
          const int nk = phase == 0 ? NK1 : NK2;
          for (int kk = 0; kk < nk; kk++, g++) {
            const int s = (int)(g % STAGES);
            if (g >= STAGES && !mbar_wait(&S.empty[s], (uint32_t)(((g / STAGES) - 1) & 1))) {
              *abort_flag = 1;
              break;
            }
            if (phase == 0) {   // h2 and W3 (hi, and lo for the split)
              mbar_expect_tx(&S.full[s], (uint32_t)(SM::OB * (BM + L3_N1) * KB));
              tma_load_3d(S.A[s], &tmH2, &S.full[s], kk * BK, tm, trt * BM);
              tma_load_3d(S.B[s], &tmW3, &S.full[s], kk * BK, 0, tm * NE + te);
              if (SPLIT) {
                tma_load_3d(S.A[s] + BM * KB, &tmH2_lo, &S.full[s], kk * BK, tm, trt * BM);
                tma_load_3d(S.B[s] + L3_N1 * KB, &tmW3_lo, &S.full[s], kk * BK, 0, tm * NE + te);
              }
            } else {            // W3^T (hi, lo)
              mbar_expect_tx(&S.full[s], (uint32_t)(SM::OB * L3_N2 * KB));
              tma_load_3d(S.B[s], &tmW3T, &S.full[s], kk * BK, 0, tm * NE + te);
              if (SPLIT) tma_load_3d(S.B[s] + L3_N2 * KB, &tmW3T_lo, &S.full[s], kk * BK, 0, tm * NE + te);
            }
            issued = g + 1;
          }
          if (*abort_flag) break;
        }
        if (!have) break;
        prev = t;
      }
      for (long long q = (issued > STAGES ? issued - STAGES : 0); q < issued; q++)
        if (!mbar_wait(&S.full[q % STAGES], (uint32_t)((q / STAGES) & 1))) *abort_flag = 1;
    }
  } else if (warp == 1) {
    if (lane == 0) {  // ---- MMA issuer
      const uint32_t id1 = idesc_bf16(BM, L3_N1), id2 = idesc_bf16(BM, L3_N2);
      const uint32_t gacc = tmem + (uint32_t)L3_GCOL;
      long long g = 0;
      int k = 0;   // valid tiles of this CTA seen so far
      bool more = true;
      for (int t = blockIdx.x; more && !*abort_flag; t += gridDim.x) {
        int rt, m, e;
        const bool have = t < T;
        if (have && !l3_tile(p, t, rt, m, e)) continue;
        more = have;
        // G1(k) into Z[k & 1]: G2(k - 2), which read that region as its A, must be complete
        if (have) {
          if (k >= 2 && !mbar_wait(&S.g_full, (uint32_t)((k - 2) & 1))) {
            *abort_flag = 1;
            break;
          }
          fence_after();
          const uint32_t z = tmem + (uint32_t)((k & 1) * L3_ZCOLS);
          for (int kb = 0; kb < NK1; kb++, g++) {
            const int s = (int)(g % STAGES);
            if (!mbar_wait(&S.full[s], (uint32_t)((g / STAGES) & 1))) {
              *abort_flag = 1;
              break;
            }
            fence_after();
            const uint32_t a0 = smem_u32(S.A[s]), b0 = smem_u32(S.B[s]);
#pragma unroll
            for (int q = 0; q < KB / 32; q++) {
              const uint64_t ah = sdesc<KB>(a0 + 32 * q), bh = sdesc<KB>(b0 + 32 * q);
              mma_bf16(z, ah, bh, id1, (kb | q) != 0);
              if (SPLIT) {   // + hi lo + lo hi
                mma_bf16(z, ah, sdesc<KB>(b0 + L3_N1 * KB + 32 * q), id1, 1u);
                mma_bf16(z, sdesc<KB>(a0 + BM * KB + 32 * q), bh, id1, 1u);
              }
            }
            mma_commit(&S.empty[s]);
          }
          if (*abort_flag) break;
          mma_commit(&S.z_full[k & 1]);
        }
        // G2(k - 1): A = g3 of tile k - 1 in Z[(k - 1) & 1] once E1 wrote it; G free once E2(k - 2) read it
        if (k >= 1) {
          const int j = k - 1;
          if (!mbar_wait(&S.a_full[j & 1], (uint32_t)((j >> 1) & 1)) ||
              (j >= 1 && !mbar_wait(&S.g_empty, (uint32_t)((j - 1) & 1)))) {
            *abort_flag = 1;
            break;
          }
          fence_after();
          const uint32_t za = tmem + (uint32_t)((j & 1) * L3_ZCOLS);
          bool first = true;
          for (int kk = 0; kk < NK2; kk++, g++) {
            const int s = (int)(g % STAGES);
            if (!mbar_wait(&S.full[s], (uint32_t)((g / STAGES) & 1))) {
              *abort_flag = 1;
              break;
            }
            fence_after();
            const uint32_t b0 = smem_u32(S.B[s]);
#pragma unroll
            for (int q = 0; q < KB / 32; q++) {
              const int kblk = kk * (BK / 16) + q;   // 16-element K block of g3
              if (16 * kblk >= L3_K2) continue;
              const uint32_t ah = za + (uint32_t)(16 * kblk);
              const uint64_t bh = sdesc<KB>(b0 + 32 * q);
              mma_bf16_ts(gacc, ah, bh, id2, first ? 0u : 1u);
              if (SPLIT) {   // + hi lo + lo hi
                mma_bf16_ts(gacc, ah, sdesc<KB>(b0 + L3_N2 * KB + 32 * q), id2, 1u);
                mma_bf16_ts(gacc, ah + 8u, bh, id2, 1u);
              }
              first = false;
            }
            mma_commit(&S.empty[s]);
          }
          if (*abort_flag) break;
          mma_commit(&S.g_full);
        }
        if (have) k++;
      }
      mma_commit(&S.fin);
      if (!mbar_wait(&S.fin, 0)) *abort_flag = 1;
    }
  } else {  // ---- epilogue warps
    const int q = warp & 3;
    const int part = (warp - 2) >> 2;
    const int r = q * 32 + lane;
    const int ew = warp - 2;
    constexpr int PB = 32 * 32;
    constexpr int NAUX = SM::NAUX;
    uint8_t *wb = S.O + (size_t)ew * NAUX * SM::OB * SM::WBUF;
    uint32_t aux_phase[NAUX];
    for (int i = 0; i < NAUX; i++) aux_phase[i] = 0u;
    unsigned aux_out = 0;      // lane 0: buffers with a load not yet consumed
    auto load_aux = [&](int b, int col, int rt, int m) {
      uint8_t *ob = wb + (size_t)b * SM::OB * SM::WBUF;
      mbar_expect_tx(&S.aux_bar[ew][b], (uint32_t)(SPLIT ? 2 * PB : PB));
      tma_load_3d(ob, &tmX, &S.aux_bar[ew][b], col, m, rt * BM + q * 32);
      if (SPLIT) tma_load_3d(ob + SM::WBUF, &tmX_lo, &S.aux_bar[ew][b], col, m, rt * BM + q * 32);
      aux_out |= 1u << b;
    };
    int k = 0;
    int prev = -1;
    bool more = true, abort_now = false;
    for (int t = blockIdx.x; more && !abort_now; t += gridDim.x) {
      int rt, m, e;
      const bool have = t < T;
      if (have && !l3_tile(p, t, rt, m, e)) continue;
      more = have;
      int prt = 0, pm = 0, pe = 0;
      if (k >= 1) l3_tile(p, prev, prt, pm, pe);
      // aux rows (h2) of the first NAUX E2(k - 1) pieces of this warp, in flight while E1(k) runs; the
      // buffers' previous stores (E2(k - 2)) must have finished reading them
      if (k >= 1 && lane == 0) {
        bulk_wait_read0();
        for (int i = 0; i < NAUX; i++) load_aux(i, 16 * part + 64 * i, prt, pm);
      }
      if (have) {  // ---- E1(k): z3 -> y partials and g3 (bf16 pairs, in place)
        // b3 and w4 of this warp's pieces, one value per lane (lanes 0-15 b3, 16-31 w4), broadcast by shuffles
        const size_t wo = ((size_t)m * NE + e) * L3_N1 + (lane & 15);
        const float *src = lane < 16 ? p.b3 : p.w4;
        float pre[3];
#pragma unroll
        for (int i = 0; i < 3; i++) {
          const int c = 16 * part + 64 * i;
          pre[i] = c < L3_N1 ? __ldg(src + wo + c) : 0.f;
        }
        if (!__all_sync(0xffffffffu, mbar_wait(&S.z_full[k & 1], (uint32_t)((k >> 1) & 1)))) {
          abort_now = true;
          break;
        }
        fence_after();
        const uint32_t zb = tmem + (uint32_t)((k & 1) * L3_ZCOLS) + ((uint32_t)(q * 32) << 16);
        float ysum = 0.f;
#pragma unroll
        for (int i = 0; i < 3; i++) {
          const int c = 16 * part + 64 * i;
          if (c >= L3_N1) break;   // warp-uniform
          float v[16];
          tmem_ld16(zb + c, v);
          uint32_t pk[16];
#pragma unroll
          for (int jj = 0; jj < 8; jj++) {   // column pair (2 jj, 2 jj + 1) -> hi and lo words
            float g[2];
#pragma unroll
            for (int u = 0; u < 2; u++) {
              const float z = v[2 * jj + u] + __shfl_sync(0xffffffffu, pre[i], 2 * jj + u);
              const float w = __shfl_sync(0xffffffffu, pre[i], 16 + 2 * jj + u);
              const float ez = exp2_approx(fminf(z, 0.f) * (CELU_INV_ALPHA * LOG2E));   // exp(min(z, 0) / alpha)
              const bool pos = z > 0.f;
              ysum = fmaf(pos ? z : fmaf(CELU_ALPHA, ez, -CELU_ALPHA), w, ysum);
              g[u] = (p.scale * w) * (pos ? 1.f : ez);
            }
            const __nv_bfloat162 hi = __floats2bfloat162_rn(g[0], g[1]);
            const float2 hf = __bfloat1622float2(hi);
            const __nv_bfloat162 lo = __floats2bfloat162_rn(g[0] - hf.x, g[1] - hf.y);
            pk[jj] = *reinterpret_cast<const uint32_t *>(&hi);
            pk[8 + jj] = *reinterpret_cast<const uint32_t *>(&lo);
          }
          tmem_st16(zb + c, pk);
        }
        tmem_wait_st();
        p.ypart[(((long long)rt * BM + r) * p.M + m) * 4 + part] = ysum;
        fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&S.a_full[k & 1]);
      }
      if (k >= 1) {  // ---- E2(k - 1): (g3 W3) * CELU'(h2) -> g2
        if (!__all_sync(0xffffffffu, mbar_wait(&S.g_full, (uint32_t)((k - 1) & 1)))) {
          abort_now = true;
          break;
        }
        fence_after();
        const uint32_t gb = tmem + (uint32_t)L3_GCOL + ((uint32_t)(q * 32) << 16);
#pragma unroll 1
        for (int i = 0; i < L3_PIECES; i++) {
          const int c = 16 * part + 64 * i;
          const int b = i % NAUX;
          float v[16];
          tmem_ld16(gb + c, v);
          uint8_t *ob = wb + (size_t)b * SM::OB * SM::WBUF;
          const bool got = mbar_wait(&S.aux_bar[ew][b], aux_phase[b]);
          aux_phase[b] ^= 1u;
          if (lane == 0) aux_out &= ~(1u << b);
          if (!__all_sync(0xffffffffu, got)) {
            abort_now = true;
            break;
          }
#pragma unroll
          for (int h8 = 0; h8 < 2; h8++) {   // eight columns at a time: aux in, g2 (hi, lo) out, in place
            uint8_t *hp = ob + lane * 32 + 16 * h8;
            alignas(16) __nv_bfloat162 ha[4], hl[4];
            *reinterpret_cast<uint4 *>(ha) = *reinterpret_cast<const uint4 *>(hp);
            if (SPLIT) *reinterpret_cast<uint4 *>(hl) = *reinterpret_cast<const uint4 *>(hp + SM::WBUF);
#pragma unroll
            for (int jj = 0; jj < 4; jj++) {
              float2 h = __bfloat1622float2(ha[jj]);
              if (SPLIT) {
                const float2 l = __bfloat1622float2(hl[jj]);
                h.x += l.x;
                h.y += l.y;
              }
              const float f0 = v[8 * h8 + 2 * jj] * dcelu_h(h.x), f1 = v[8 * h8 + 2 * jj + 1] * dcelu_h(h.y);
              ha[jj] = __floats2bfloat162_rn(f0, f1);
              if (SPLIT) {
                const float2 hi = __bfloat1622float2(ha[jj]);
                hl[jj] = __floats2bfloat162_rn(f0 - hi.x, f1 - hi.y);
              }
            }
            *reinterpret_cast<uint4 *>(hp) = *reinterpret_cast<const uint4 *>(ha);
            if (SPLIT) *reinterpret_cast<uint4 *>(hp + SM::WBUF) = *reinterpret_cast<const uint4 *>(hl);
          }
          fence_proxy_async();
          __syncwarp();
          if (lane == 0) {
            tma_store_3d(&tmO, ob, c, pm, prt * BM + q * 32);
            if (SPLIT) tma_store_3d(&tmO_lo, ob + SM::WBUF, c, pm, prt * BM + q * 32);
            bulk_commit();
            if (i + NAUX < L3_PIECES) {   // a later piece reuses this buffer once the store has read it
              bulk_wait_read0();
              load_aux(b, c + 64 * NAUX, prt, pm);
            }
          }
        }
        if (abort_now) break;
        fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&S.g_empty);
      }
      if (have) {
        prev = t;
        k++;
      }
    }
    if (abort_now) *abort_flag = 1;
    if (lane == 0) {
      bulk_wait_all();
      for (int i = 0; i < NAUX; i++)   // loads issued and not consumed: let them land before the CTA exits
        if ((aux_out >> i) & 1u)
          if (!mbar_wait(&S.aux_bar[ew][i], aux_phase[i])) *abort_flag = 1;
    }
  }
  fence_before();
  __syncthreads();
  if (*abort_flag && threadIdx.x == 0) post_status(p.st, FNN_E_TIMEOUT, blockIdx.x);
  if (warp == 1) {
    fence_after();
    tmem_dealloc(tmem, 2 * TMEM_COLS);
  }
}

}  // namespace tc
}  // namespace fnn
