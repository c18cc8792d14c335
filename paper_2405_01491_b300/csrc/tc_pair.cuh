// Two-SM (cta_group::2) form of the first layer's products (section II.B), sm_103a: the forward
// h1 = CELU(aev W1cat^T + b1) (EPI_BIAS_CELU; bf16, split or e4m3 operands) and the input gradient
// dE/dAEV = g1 W1cat (EPI_F32; N = 1008 in four 256-column n tiles, fp32 out).
//
// A cluster of two CTAs (one SM each) computes a 256 x 256 tile: two 128-row tiles of one element's
// species-sorted AEV rows against one member's 256 first-layer outputs.  Each CTA stages its own 128 A
// rows and half of the member's weight rows (128 of the 256 output columns); one thread of the even CTA
// issues tcgen05.mma with M = 256, which reads both CTAs' shared memory and writes each CTA's TMEM with
// its own 128 rows x 256 columns.  Per SM this is the work of the one-SM tile for two thirds of its operand
// bytes: the one-SM first layer is bound by the rate at which an SM stages operand bytes from L2 (41-51
// bytes per cycle measured), and a stage here is 64 KB (split: hi and lo of both operands) instead of 96 KB,
// so three stages fit where two
// did (bf16 and e4m3: 32 KB instead of 48, six stages).  The partial last wave's items are cut into two
// column halves (N = 128) when there are clusters for all of them, or, for the fp32 input gradient, along K
// into parts added by TMA reduce-add into tiles a side-stream kernel zeroed (its schedule is pair_tail_sched).
//   warp 0 (one lane, both CTAs)  TMA producer: its A rows and B half into its own ring, completion counted
//                                 on the even CTA's stage barrier (the pair's expected bytes set there)
//   warp 1 (both CTAs)            TMEM allocation for the pair; one lane of the even CTA issues the MMAs and
//                                 commits each stage's release and each accumulator to both CTAs' barriers
//   warps 2-17 (both CTAs)        bias + CELU (or fp32) epilogue of the CTA's own rows (as the one-SM kernel),
//                                 then an arrival on the even CTA's accumulator-free barrier
// Pairs are two consecutive row tiles of one element; an element with an odd number of row tiles ends in a
// pair whose second tile is absent (that CTA loads the first tile's rows again and stores nothing).
// Every mbarrier wait is bounded; on timeout the CTA posts FNN_E_TIMEOUT and both CTAs meet at the final
// cluster barrier before TMEM is released.
#pragma once

#include "tc_gemm.cuh"

namespace fnn {
namespace tc {

// ---------------------------------------------------------------------------------- cluster pairs
__device__ __forceinline__ uint32_t pair_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
// the shared::cluster address of a shared-memory location of this CTA in the pair's CTA `rank`
__device__ __forceinline__ uint32_t pair_addr(const void *p, uint32_t rank) {
  uint32_t d;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(d) : "r"(smem_u32(p)), "r"(rank));
  return d;
}
__device__ __forceinline__ void pair_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
// arrive on an mbarrier of either CTA of the pair (release at cluster scope)
__device__ __forceinline__ void mbar_arrive_remote(uint32_t caddr) {
  asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(caddr) : "memory");
}
// bounded wait with acquire at cluster scope (arrivals from the other CTA of the pair)
__device__ __forceinline__ bool mbar_try_wait_cl(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ bool mbar_wait_cl(uint64_t *bar, uint32_t parity) {
  if (mbar_try_wait_cl(bar, parity)) return true;
  long long t0 = clock64();
  while (!mbar_try_wait_cl(bar, parity))
    if (clock64() - t0 > WAIT_LIMIT) return false;
  return true;
}
// TMA load into this CTA's shared memory, its bytes counted on an mbarrier of either CTA of the pair
__device__ __forceinline__ void tma_load_3d_pair(void *dst, const CUtensorMap *map, uint32_t bar_cl, int c0, int c1,
                                                 int c2) {
  asm volatile(
      "cp.async.bulk.tensor.3d.cta_group::2.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, "
      "%5}], [%2];" ::"r"(smem_u32(dst)),
      "l"((uint64_t)map), "r"(bar_cl), "r"(c0), "r"(c1), "r"(c2)
      : "memory");
}
// TMEM of the pair: executed by one warp of each CTA
__device__ __forceinline__ void tmem_alloc_pair(uint32_t *dst, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst)), "r"(ncols)
               : "memory");
}
__device__ __forceinline__ void tmem_relinquish_pair() {
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc_pair(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
// D (each CTA's TMEM, its 128 rows) (+)= A (both CTAs' 128 rows) * B (both CTAs' N / 2 rows)^T
__device__ __forceinline__ void mma_bf16_pair(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc));
}
// the same with e4m3 operands (kind::f8f6f4, fp32 accumulation)
__device__ __forceinline__ void mma_f8_pair(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::2.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc));
}
// arrive on the mbarrier at this offset in both CTAs of the pair once this thread's MMAs have completed
__device__ __forceinline__ void mma_commit_pair(uint64_t *bar) {
  asm volatile(
      "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;" ::"r"(
          smem_u32(bar)),
      "h"((uint16_t)3)
      : "memory");
}
// the same, on this CTA's mbarrier only
__device__ __forceinline__ void mma_commit_pair_local(uint64_t *bar) {
  asm volatile("tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

// ---------------------------------------------------------------------------------- kernel
constexpr int PAIR_NT = 256;          // output columns of a tile (one member's first layer)
constexpr int PAIR_NH = PAIR_NT / 2;  // weight rows staged per CTA

struct PairArgs {
  int K;                       // reduction length (1008)
  int n_nt;                    // n tiles: members (output column block nt * 256)
  const int32_t *meta;         // META_SEG: padded row starts of the elements (multiples of 128)
  const float *bias;           // bias + e * bias_estride + nt * 256 + c
  long long bias_estride;
  DevStatus *st;
  // fp8 (MODE_F8): A = a8 * a_scale, B = b8 * b_scale[nt * 7 + e]; the output holds x * out_inv
  float a_scale, out_inv;
  const float *b_scale;
  // EPI_F32 (the input gradient dE/dAEV = g1 W1cat): N valid output columns of the product, stored through
  // the output map (32-row x 8-column fp32 boxes) at x = nt 256 + c; with tail_split the partial wave is cut
  // along K and added into tiles zeroed beforehand
  int N, tail_split;
};

template <int MODE, int EPI = EPI_BIAS_CELU>
struct PairSmem {
  static constexpr bool SPLIT = MODE == MODE_SPLIT;
  // (rows of 128 bytes: 64 bf16 or 128 e4m3 elements of K)
  static constexpr int AQ = SPLIT ? 2 : 1;                 // hi and lo of each operand per stage
  // output halves per buffer and buffers per epilogue warp (fp32 pieces of 32 rows x 8 columns: two buffers)
  static constexpr int OB = (SPLIT && EPI != EPI_F32) ? 2 : 1;
  static constexpr int NBUF = (SPLIT && EPI != EPI_F32) ? 1 : 2;
  static constexpr int WBUF = 1024;                        // 32 rows x 16 bf16 (or 8 fp32) columns
  static constexpr int OBYTES = EPI_WARPS * NBUF * OB * WBUF;
  static constexpr int STAGE = AQ * (BM + PAIR_NH) * BKB;  // this CTA's bytes of one K chunk
  static constexpr int FIT = (SMEM_LIMIT - 1024 - OBYTES - 1024) / STAGE;
  static constexpr int STAGES = FIT > 6 ? 6 : FIT;
  uint8_t A[STAGES][AQ * BM * BKB];
  uint8_t B[STAGES][AQ * PAIR_NH * BKB];
  uint8_t O[OBYTES];
  uint64_t full[STAGES], empty[STAGES], acc_full[2], acc_empty[2], fin;
  uint32_t tmem_base;
  int abort_flag;
};
template <int MODE, int EPI = EPI_BIAS_CELU>
constexpr size_t pair_smem_bytes() {
  return sizeof(PairSmem<MODE, EPI>) + 1024;
}

// item t of the pair schedule -> (n tile, the pair's first row tile, element, whether its second tile
// exists); false past the last item.  Items run n tile fastest, then pairs in element order.
__device__ __forceinline__ bool pair_item(const int seg[NE + 1], int n_nt, int t, int &nt, int &rt0, int &e,
                                          bool &two) {
  nt = t % n_nt;
  int j = t / n_nt;
  for (e = 0; e < NE; e++) {
    const int t0 = seg[e] / BM, t1 = seg[e + 1] / BM, np = (t1 - t0 + 1) / 2;
    if (j < np) {
      rt0 = t0 + 2 * j;
      two = rt0 + 1 < t1;
      return true;
    }
    j -= np;
  }
  return false;
}

// Work item `it` of cluster cl among ncl: the T items' whole waves, then the R items of the partial wave.
// Bias + CELU products cut those into two column halves (N = 128, each CTA staging 64 weight rows) when
// there are clusters for all halves; fp32 products (ksplit) cut them along K into S = min(ncl / R, nkb)
// parts, part cl % S of item W ncl + cl / S going to cluster cl < R S and added into its tile (zeroed
// beforehand, pair_tail_sched).
struct PairWork {
  int nt, rt0, e, c0, cw, kb0, kb1;
  bool two, atomic;
};
struct PairTail {
  int W, R, S;
};
__device__ __forceinline__ PairTail pair_tail_sched(int T, int ncl, int nkb) {
  PairTail s;
  s.W = T / ncl;
  s.R = T - s.W * ncl;
  s.S = s.R ? min(ncl / s.R, nkb) : 0;
  return s;
}
__device__ __forceinline__ bool pair_work(const int seg[NE + 1], int n_nt, int T, int cl, int ncl, int it, PairWork &w,
                                          bool ksplit = false, int nkb = 0) {
  const int W = T / ncl, R = T - W * ncl;
  int t;
  w.c0 = 0;
  w.cw = PAIR_NT;
  w.kb0 = 0;
  w.kb1 = nkb;
  w.atomic = false;
  if (ksplit && R > 0) {
    const PairTail ts = pair_tail_sched(T, ncl, nkb);
    if (it < W) {
      t = cl + it * ncl;
    } else if (it == W && cl < ts.R * ts.S) {
      const int part = cl % ts.S;
      t = W * ncl + cl / ts.S;
      w.kb0 = part * nkb / ts.S;
      w.kb1 = (part + 1) * nkb / ts.S;
      w.atomic = true;
    } else {
      return false;
    }
  } else if (ksplit || R == 0 || 2 * R > ncl) {
    t = cl + it * ncl;
    if (t >= T) return false;
  } else if (it < W) {
    t = cl + it * ncl;
  } else if (it == W && cl < 2 * R) {
    t = W * ncl + cl / 2;
    w.c0 = (cl & 1) * (PAIR_NT / 2);
    w.cw = PAIR_NT / 2;
  } else {
    return false;
  }
  return pair_item(seg, n_nt, t, w.nt, w.rt0, w.e, w.two);
}

template <int MODE, int EPI = EPI_BIAS_CELU>
__global__ void __launch_bounds__(THREADS, 1)
    k_umma_pair(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmA_lo,
                const __grid_constant__ CUtensorMap tmB, const __grid_constant__ CUtensorMap tmB_lo,
                const __grid_constant__ CUtensorMap tmO, const __grid_constant__ CUtensorMap tmO_lo, PairArgs p) {
  static_assert(MODE == MODE_SPLIT || MODE == MODE_BF16 || MODE == MODE_F8, "bf16, its three-term split, or e4m3");
  static_assert(EPI == EPI_BIAS_CELU || (EPI == EPI_F32 && MODE != MODE_F8), "bias + CELU, or the fp32 input gradient");
  using SM = PairSmem<MODE, EPI>;
  constexpr bool F32 = EPI == EPI_F32;
  static_assert(SM::STAGES >= 2 && sizeof(SM) + 1024 <= SMEM_LIMIT, "shared memory budget");
  constexpr bool SPLIT = SM::SPLIT, F8 = MODE == MODE_F8;
  constexpr int STAGES = SM::STAGES, KB = BKB, BK = F8 ? KB : KB / 2;   // K elements per stage
  extern __shared__ uint8_t smem_raw[];
  SM &S = *reinterpret_cast<SM *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t rank = pair_rank();
  const bool leader = rank == 0;
  const int cl = (int)blockIdx.x >> 1, ncl = (int)gridDim.x >> 1;
  const int nkb = (p.K + BK - 1) / BK;
  volatile int *abort_flag = &S.abort_flag;
  int seg[NE + 1];
#pragma unroll
  for (int e = 0; e <= NE; e++) seg[e] = p.meta[META_SEG + e];
  int T = 0;   // items: n tiles x row-tile pairs
#pragma unroll
  for (int e = 0; e < NE; e++) T += (seg[e + 1] / BM - seg[e] / BM + 1) / 2;
  T *= p.n_nt;
  const bool ksplit = F32 && p.tail_split;

  if (warp == 0 && lane == 0) {
    for (int s = 0; s < STAGES; s++) {
      mbar_init(&S.full[s], 1);
      mbar_init(&S.empty[s], 1);
    }
    for (int a = 0; a < 2; a++) {
      mbar_init(&S.acc_full[a], 1);
      mbar_init(&S.acc_empty[a], 2 * EPI_WARPS);   // every epilogue warp of both CTAs
    }
    mbar_init(&S.fin, 1);
    S.abort_flag = 0;
    fence_barrier_init();
  }
  if (warp == 1) {
    tmem_alloc_pair(&S.tmem_base, 2 * TMEM_COLS);
    tmem_relinquish_pair();
  }
  fence_before();
  __syncthreads();
  pair_sync();   // both CTAs' barriers initialised before either signals the other's
  fence_after();
  const uint32_t tmem = S.tmem_base;

  if (warp == 0) {
    if (lane == 0) {  // ---- TMA producer (both CTAs)
      long long g = 0;
      long long issued = 0;
      for (int it = 0; !*abort_flag; it++) {
        PairWork w;
        if (!pair_work(seg, p.n_nt, T, cl, ncl, it, w, ksplit, nkb)) break;
        const int rt = (rank == 1 && w.two) ? w.rt0 + 1 : w.rt0;   // an absent second tile reloads the first's rows
        const int bh = w.cw / 2;                                    // weight rows staged by this CTA
        const int by = w.nt * PAIR_NT + w.c0 + (int)rank * bh;
        for (int kb = w.kb0; kb < w.kb1; kb++, g++) {
          const int s = (int)(g % STAGES);
          if (g >= STAGES && !mbar_wait(&S.empty[s], (uint32_t)(((g / STAGES) - 1) & 1))) {
            *abort_flag = 1;
            break;
          }
          const uint32_t fb = pair_addr(&S.full[s], 0);
          if (leader) mbar_expect_tx(&S.full[s], (uint32_t)(2 * SM::AQ * (BM + bh) * KB));
          tma_load_3d_pair(S.A[s], &tmA, fb, kb * BK, 0, rt * BM);
          if (SPLIT) tma_load_3d_pair(S.A[s] + BM * KB, &tmA_lo, fb, kb * BK, 0, rt * BM);
          // the weight rows: 64-row boxes (8-row swizzle groups, so stacked boxes form one taller tile)
          for (int h = 0; h < bh; h += 64) {
            tma_load_3d_pair(S.B[s] + h * KB, &tmB, fb, kb * BK, by + h, w.e);
            if (SPLIT) tma_load_3d_pair(S.B[s] + PAIR_NH * KB + h * KB, &tmB_lo, fb, kb * BK, by + h, w.e);
          }
          issued = g + 1;
        }
      }
      // drain (the even CTA, whose stage barriers count both CTAs' bytes): every issued load lands before
      // the pair can leave its final cluster barrier
      if (leader)
        for (long long q = (issued > STAGES ? issued - STAGES : 0); q < issued; q++)
          if (!mbar_wait(&S.full[q % STAGES], (uint32_t)((q / STAGES) & 1))) *abort_flag = 1;
    }
  } else if (warp == 1) {
    if (lane == 0 && leader) {  // ---- MMA issuer (the even CTA)
      long long g = 0;
      int cnt = 0;
      for (int it = 0; !*abort_flag; it++) {
        PairWork w;
        if (!pair_work(seg, p.n_nt, T, cl, ncl, it, w, ksplit, nkb)) break;
        const uint32_t idesc = F8 ? idesc_e4m3(2 * BM, w.cw) : idesc_bf16(2 * BM, w.cw);
        const int a = cnt & 1;
        if (cnt >= 2 && !mbar_wait_cl(&S.acc_empty[a], (uint32_t)(((cnt >> 1) - 1) & 1))) {
          *abort_flag = 1;
          break;
        }
        fence_after();
        const uint32_t d = tmem + (uint32_t)(a * TMEM_COLS);
        for (int kb = w.kb0; kb < w.kb1; kb++, g++) {
          const int s = (int)(g % STAGES);
          if (!mbar_wait(&S.full[s], (uint32_t)((g / STAGES) & 1))) {
            *abort_flag = 1;
            break;
          }
          fence_after();
          const uint32_t a0 = smem_u32(S.A[s]), b0 = smem_u32(S.B[s]);
#pragma unroll
          for (int k = 0; k < KB / 32; k++) {
            const uint32_t acc = (kb != w.kb0 || k != 0) ? 1u : 0u;   // the item's first K step starts the sum
            if (SPLIT) {   // hi hi + hi lo + lo hi of this K step
              const uint64_t ah = sdesc_sw128(a0 + 32 * k), al = sdesc_sw128(a0 + BM * KB + 32 * k);
              const uint64_t bh = sdesc_sw128(b0 + 32 * k), bl = sdesc_sw128(b0 + PAIR_NH * KB + 32 * k);
              mma_bf16_pair(d, ah, bh, idesc, acc);
              mma_bf16_pair(d, ah, bl, idesc, 1u);
              mma_bf16_pair(d, al, bh, idesc, 1u);
            } else if (F8) {
              mma_f8_pair(d, sdesc_sw128(a0 + 32 * k), sdesc_sw128(b0 + 32 * k), idesc, acc);
            } else {
              mma_bf16_pair(d, sdesc_sw128(a0 + 32 * k), sdesc_sw128(b0 + 32 * k), idesc, acc);
            }
          }
          mma_commit_pair(&S.empty[s]);   // stage s free in both CTAs once these MMAs finish
        }
        if (*abort_flag) break;
        mma_commit_pair(&S.acc_full[a]);   // accumulator a of both CTAs complete
        cnt++;
      }
      mma_commit_pair_local(&S.fin);
      if (!mbar_wait(&S.fin, 0)) *abort_flag = 1;
    }
  } else {  // ---- epilogue warps 2 .. 2 + EPI_WARPS - 1 (both CTAs, each its own 128 rows)
    const int q = warp & 3;                 // TMEM lane quarter this warp may read
    const int part = (warp - 2) >> 2;       // which of the quarter's four warps: chunks part, part + 4, ...
    const int ew = warp - 2;
    uint8_t *wb = S.O + (size_t)ew * SM::NBUF * SM::OB * SM::WBUF;
    const uint32_t empty0 = pair_addr(&S.acc_empty[0], 0), empty1 = pair_addr(&S.acc_empty[1], 0);
    long long gk = 0;
    int cnt = 0;
    for (int it = 0;; it++) {
      PairWork w;
      if (!pair_work(seg, p.n_nt, T, cl, ncl, it, w, ksplit, nkb)) break;
      const bool mine = rank == 0 || w.two;   // this CTA's tile exists
      const int rt = rank == 1 ? w.rt0 + 1 : w.rt0, nt = w.nt;
      const int a = cnt & 1;
      const int npc = w.cw / 64;              // this warp's 16-column pieces of the item
      // the bias of this warp's pieces (lane j: column j of piece i), read while the MMAs run
      const float *bias = p.bias + w.e * p.bias_estride + nt * PAIR_NT + w.c0;
      float pre[PAIR_NT / 64];
#pragma unroll
      for (int i = 0; i < PAIR_NT / 64; i++)
        pre[i] = (!F32 && i < npc) ? __ldg(bias + 16 * part + 64 * i + (lane & 15)) : 0.f;
      const float sc = F8 ? p.a_scale * p.b_scale[nt * NE + w.e] : 1.f;   // dequantisation of the fp8 product
      const bool ok = mbar_wait(&S.acc_full[a], (uint32_t)((cnt >> 1) & 1));
      fence_after();
      if (!__all_sync(0xffffffffu, ok)) {
        *abort_flag = 1;
        break;
      }
      const uint32_t tbase = tmem + (uint32_t)(a * TMEM_COLS) + ((uint32_t)(q * 32) << 16);
      if (mine && F32) {
        // 32-row x 8-column fp32 pieces through this warp's two buffers, stored by TMA, or for a K part of a
        // tail tile added into the tile zeroed beforehand; columns at or beyond N are not written
        const int ncols = min(w.cw, p.N - nt * PAIR_NT - w.c0);
#pragma unroll 1
        for (int i = 0; i < npc; i++) {
          const int c = 16 * part + 64 * i;
          if (c >= ncols) break;   // warp-uniform; ncols is a multiple of 16
          float v[16];
          tmem_ld16(tbase + c, v);
#pragma unroll
          for (int hh = 0; hh < 2; hh++) {
            uint8_t *ob = wb + (size_t)(gk & 1) * SM::WBUF;
            if (lane == 0 && gk >= 2) bulk_wait_read1();   // the operation that last read this buffer
            __syncwarp();
            float4 *d4 = reinterpret_cast<float4 *>(ob + lane * 32);
            d4[0] = make_float4(v[8 * hh], v[8 * hh + 1], v[8 * hh + 2], v[8 * hh + 3]);
            d4[1] = make_float4(v[8 * hh + 4], v[8 * hh + 5], v[8 * hh + 6], v[8 * hh + 7]);
            fence_proxy_async();
            __syncwarp();
            if (lane == 0) {
              const int x = nt * PAIR_NT + w.c0 + c + 8 * hh;
              if (w.atomic) tma_reduce_add_3d(&tmO, ob, x, 0, rt * BM + q * 32);
              else tma_store_3d(&tmO, ob, x, 0, rt * BM + q * 32);
              bulk_commit();
            }
            gk++;
          }
        }
      } else if (mine) {
#pragma unroll 1
        for (int i = 0; i < npc; i++) {
          const int c = 16 * part + 64 * i;   // column of the item (output column w.c0 + c)
          float v[16];
          tmem_ld16(tbase + c, v);
          uint8_t *ob = wb + (size_t)(gk % SM::NBUF) * SM::OB * SM::WBUF;
          if (lane == 0 && SM::NBUF == 2 && gk >= 2) bulk_wait_read1();
          if (lane == 0 && SM::NBUF == 1 && gk >= 1) bulk_wait_read0();
          __syncwarp();
          float f[16];
#pragma unroll
          for (int j = 0; j < 16; j++) f[j] = celu_f((F8 ? v[j] * sc : v[j]) + __shfl_sync(0xffffffffu, pre[i], j));
          if (F8) {  // saturating round-to-nearest e4m3 of x * out_inv
            alignas(16) __nv_fp8x2_storage_t q8[8];
#pragma unroll
            for (int j = 0; j < 8; j++)
              q8[j] = __nv_cvt_float2_to_fp8x2(make_float2(f[2 * j] * p.out_inv, f[2 * j + 1] * p.out_inv),
                                               __NV_SATFINITE, __NV_E4M3);
            *reinterpret_cast<uint4 *>(ob + lane * 16) = *reinterpret_cast<const uint4 *>(q8);
          } else {
            alignas(16) __nv_bfloat162 o2[8];
#pragma unroll
            for (int j = 0; j < 8; j++) o2[j] = __floats2bfloat162_rn(f[2 * j], f[2 * j + 1]);
            *reinterpret_cast<uint4 *>(ob + lane * 32) = *reinterpret_cast<const uint4 *>(o2);
            *reinterpret_cast<uint4 *>(ob + lane * 32 + 16) = *reinterpret_cast<const uint4 *>(o2 + 4);
            if (SPLIT) {  // low part: the rounding residual of the high part
#pragma unroll
              for (int j = 0; j < 8; j++) {
                const float2 hi = __bfloat1622float2(o2[j]);
                o2[j] = __floats2bfloat162_rn(f[2 * j] - hi.x, f[2 * j + 1] - hi.y);
              }
              *reinterpret_cast<uint4 *>(ob + SM::WBUF + lane * 32) = *reinterpret_cast<const uint4 *>(o2);
              *reinterpret_cast<uint4 *>(ob + SM::WBUF + lane * 32 + 16) = *reinterpret_cast<const uint4 *>(o2 + 4);
            }
          }
          fence_proxy_async();
          __syncwarp();
          if (lane == 0) {
            tma_store_3d(&tmO, ob, w.c0 + c, nt, rt * BM + q * 32);
            if (SPLIT) tma_store_3d(&tmO_lo, ob + SM::WBUF, w.c0 + c, nt, rt * BM + q * 32);
            bulk_commit();
          }
          gk++;
        }
      }
      // accumulator a of the pair may be overwritten once every epilogue warp of both CTAs has read it
      fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive_remote(a ? empty1 : empty0);
      cnt++;
    }
    if (lane == 0) bulk_wait_all();   // nothing may still read this warp's buffers when the CTA exits
  }
  fence_before();
  __syncthreads();
  pair_sync();   // the pair's MMAs, remote arrivals and loads are over before TMEM is released
  if (*abort_flag && threadIdx.x == 0) post_status(p.st, FNN_E_TIMEOUT, blockIdx.x);
  if (warp == 1) {
    fence_after();
    tmem_dealloc_pair(tmem, 2 * TMEM_COLS);
  }
}

}  // namespace tc
}  // namespace fnn
