// tcgen05 (5th-generation tensor core) GEMM for the per-element networks, sm_103a.
//
// One CTA computes a 128 x NT tile C = A B^T of a "TN" product (both operands K-contiguous):
//   warp 0 (one lane)  TMA producer: 128 x 128-byte A and NT x 128-byte B tiles (64 bf16 or 128 fp8
//                      e4m3 elements of K), 128-byte swizzle, STAGES-deep ring guarded by mbarriers
//   warp 1 (one lane)  MMA issuer: 4 x tcgen05.mma (32 bytes of K each: kind::f16 K = 16, or
//                      kind::f8f6f4 K = 32) per stage, accumulator in TMEM (128 lanes x NT fp32
//                      columns); tcgen05.commit frees the stage
//   warps 2-17         epilogue: tcgen05.ld 32 lanes x 16 columns at a time (warp w reads TMEM lane
//                      quarter w % 4; the four warps of a quarter take every fourth 16-column chunk),
//                      fused bias/CELU, CELU', output-layer dot, store
// Persistent: one CTA per SM walks the tile grid; two TMEM accumulators overlap the epilogue of one
// tile with the MMAs of the next.  Every mbarrier wait is bounded; on timeout the CTA posts
// FNN_E_TIMEOUT, drains what it issued, frees its TMEM and returns.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include "fnn_internal.cuh"

namespace fnn {
namespace tc {

constexpr int BM = 128;         // rows per tile (UMMA M)
constexpr int SMEM_LIMIT = 232448;   // dynamic shared memory per block (227 KB)
constexpr int BKB = 128;        // K bytes per stage: one 128-byte swizzle row (64 bf16, 128 fp8)
constexpr int TMEM_COLS = 256;  // accumulator columns allocated (NT <= 256)
constexpr int EPI_WARPS = 16;   // four per TMEM lane quarter
constexpr int THREADS = 64 + 32 * EPI_WARPS;
constexpr long long WAIT_LIMIT = 2000000000LL;  // clock64 cycles (about a second) before a wait gives up

enum { EPI_BIAS_CELU = 0, EPI_L3 = 1, EPI_DCELU = 2, EPI_F32 = 3, EPI_PLAIN = 4, EPI_ATOMIC = 5 };
// operand forms: bf16; the three-term bf16 split of an fp32 product; fp8 e4m3 with per-tensor scales;
// bf16 weight gradients (K runs over an element's rows; A and B are read feature-contiguous, MN-major)
enum { MODE_BF16 = 0, MODE_SPLIT = 1, MODE_F8 = 2, MODE_WG = 3 };

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// ---------------------------------------------------------------------------------- mbarrier
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_barrier_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// bounded wait on the phase with the given parity; false when it did not complete in time
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity) {
  if (mbar_try_wait(bar, parity)) return true;
  long long t0 = clock64();
  while (!mbar_try_wait(bar, parity))
    if (clock64() - t0 > WAIT_LIMIT) return false;
  return true;
}

// ---------------------------------------------------------------------------------- TMA
__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, uint64_t *bar, int c0, int c1,
                                            int c2) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5}], [%2];" ::"r"(
          smem_u32(dst)),
      "l"((uint64_t)map), "r"(smem_u32(bar)), "r"(c0), "r"(c1), "r"(c2)
      : "memory");
}

// ---------------------------------------------------------------------------------- tcgen05
__device__ __forceinline__ void tmem_alloc(uint32_t *dst, uint32_t ncols) {  // whole warp
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst)), "r"(ncols)
               : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {  // whole warp
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// D[tmem] (+)= A[smem] * B[smem]^T, bf16 inputs, fp32 accumulation
__device__ __forceinline__ void mma_bf16(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc));
}
// D[tmem] (+)= A[smem] * B[smem]^T, fp8 e4m3 inputs, fp32 accumulation
__device__ __forceinline__ void mma_f8(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc));
}
// arrive on an mbarrier once every previously issued tcgen05.mma of this thread has completed
__device__ __forceinline__ void mma_commit(uint64_t *bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

// ---------------------------------------------------------------------------------- TMA store
// tile [smem] -> tensor (bulk group); the source must stay untouched until wait_group.read says so
__device__ __forceinline__ void tma_store_3d(const CUtensorMap *map, const void *src, int c0, int c1, int c2) {
  asm volatile("cp.async.bulk.tensor.3d.global.shared::cta.bulk_group [%0, {%2, %3, %4}], [%1];" ::"l"(
                   (uint64_t)map),
               "r"(smem_u32(src)), "r"(c0), "r"(c1), "r"(c2)
               : "memory");
}
// tile [smem] added into the tensor (bulk group; fp32 add by the map's element type)
__device__ __forceinline__ void tma_reduce_add_3d(const CUtensorMap *map, const void *src, int c0, int c1, int c2) {
  asm volatile("cp.reduce.async.bulk.tensor.3d.global.shared::cta.add.tile.bulk_group [%0, {%2, %3, %4}], [%1];" ::"l"(
                   (uint64_t)map),
               "r"(smem_u32(src)), "r"(c0), "r"(c1), "r"(c2)
               : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
// at most one committed store group still reading its shared-memory source
__device__ __forceinline__ void bulk_wait_read1() { asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory"); }
// no committed store group still reading its source
__device__ __forceinline__ void bulk_wait_read0() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
// every committed store group complete
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
// make this thread's shared-memory writes visible to the async proxy (TMA)
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// 32 TMEM lanes x 16 consecutive fp32 columns: thread t of the warp receives lane (base + t)
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float v[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; i++) v[i] = __uint_as_float(r[i]);
}

// Shared-memory matrix descriptor: K-major operand, 128-byte swizzle, 8-row core groups 1024 B apart.
// Fields: start address >> 4 [0,14), leading byte offset >> 4 [16,30) (unused for swizzled K-major),
// stride byte offset >> 4 [32,46), descriptor version 1 at bit 46, swizzle mode 2 (128 B) at [61,64).
__device__ __forceinline__ uint64_t sdesc_sw128(uint32_t saddr) {
  uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)1 << 16;
  d |= (uint64_t)(1024 >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}
// the same for 64-byte rows with the 64-byte swizzle: 8-row groups 512 B apart, swizzle mode 4
__device__ __forceinline__ uint64_t sdesc_sw64(uint32_t saddr) {
  uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)1 << 16;
  d |= (uint64_t)(512 >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)4 << 61;
  return d;
}
// MN-major operand, 128-byte swizzle: atoms of 8 K rows x 64 MN elements (128 bytes per K row, 1024 B);
// 8-K-row groups 1024 B apart (stride byte offset), 64-element MN blocks lbo bytes apart (leading byte offset)
__device__ __forceinline__ uint64_t sdesc_mn_sw128(uint32_t saddr, uint32_t lbo) {
  uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)(1024 >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}
// descriptor of a K-major operand whose rows are KB bytes (128 or 64), swizzled to match
template <int KB>
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr) {
  static_assert(KB == 128 || KB == 64, "row width");
  return KB == 128 ? sdesc_sw128(saddr) : sdesc_sw64(saddr);
}

// Instruction descriptor, kind::f16: fp32 accumulator [4,6) = 1, A and B bf16 [7,10) = [10,13) = 1,
// both K-major (bits 15, 16 = 0), N >> 3 at [17,23), M >> 4 at [24,29).
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}
// the same with both operands MN-major (transpose bits 15 and 16)
__host__ __device__ constexpr uint32_t idesc_bf16_mn(int M, int N) { return idesc_bf16(M, N) | (1u << 15) | (1u << 16); }
// kind::f8f6f4: fp32 accumulator, A and B format E4M3 (code 0 in [7,10) and [10,13)), both K-major
__host__ __device__ constexpr uint32_t idesc_e4m3(int M, int N) {
  return (1u << 4) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// ---------------------------------------------------------------------------------- kernel
struct Args {
  int K;                       // reduction length
  int N;                       // valid output columns of the whole product
  int n_ntiles, n_rowtiles, n_members;  // tile grid: t -> (n tile fastest, row tile, member)
  int a_by_member;             // A's middle coordinate = member (else 0)
  int b_by_member;             // B's group coordinate = member * 7 + element (else element)
  const int32_t *tile_elem;    // element of each 128-row tile (-1: skip)
  // EPI_F32: fp32 output [rows][ldo] (o_mstride 0) through the output map (box 8 x 1 x 32, fp32): stored, or
  // for the K parts of a tail-split launch added by TMA reduce-add into tiles zeroed at `out` beforehand
  float *out;
  long long ldo, o_mstride;
  // every other epilogue stores 32-row x 16-column pieces through the output tensor map (box 16 x 1 x 32):
  // columns c.. of rows z.. of tile (nt, rt, m) go to x = o_xm * m + c, y = (o_y == 1: m, 2: nt, else 0);
  // EPI_DCELU reads its aux input (h of the layer) through the aux map at x = c, y = (x_y == 1: m, else 0)
  int o_xm, o_y, x_y;
  const float *bias;
  long long bias_estride, bias_mstride;
  const float *w4;             // output layer (EPI_L3)
  long long w4_estride, w4_mstride;
  float *ypart;                // [rows][M][4] (EPI_L3, column 0)
  int M;
  float scale;
  DevStatus *st;
  // fp8 (MODE_F8): A = a8 * a_scale, B = b8 * b_scale[b_scale_sel * NE + e] with sel the tile's
  // member (b_scale_by = 1), its n tile (2) or 0 (0); fp8 outputs hold x * out_inv; aux is fp8 * aux_scale
  float a_scale, out_inv, aux_scale;
  const float *b_scale;
  int b_scale_by;
  // weight gradients (MODE_WG, EPI_ATOMIC): tile t -> (i tile, o tile, row chunk, group g = 7 m + e);
  // K = rows seg[e] + chunk * kchunk .. (at most kchunk, within the element's segment), both terms
  // (A, B) then (A_lo, B_lo); the fp32 tile is added into dW[g][O][I] by TMA reduce-add through the
  // output map (dims I, O, g; box 8 x 32 x 1)
  const int32_t *seg;
  int kchunk, n_chunks;
  int b_shared;               // B has one member for all (its z coordinate is 0)
  int O;                      // rows of dW (a 32-row piece starting at or beyond O is skipped)
  // EPI_F32 only: the tiles of the final partial wave are split along K over all CTAs and their parts
  // added atomically into the output, which the caller zeroes first (tail_sched gives the tiles)
  int tail_split;
  const int32_t *meta;         // META_NPAD bounds the valid row tiles when tail_split or tail_nsplit is set
  // other epilogues: the partial wave's tiles are cut into NT / nsub_w column strips (when there are CTAs
  // for all of them), B read through the map with nsub_w-row boxes
  int tail_nsplit, nsub_w;
};

// Persistent schedule of a tail-split launch over the valid tiles (row tiles below META_NPAD), grid G:
// CTA c takes tiles c, c + G, ... for the W whole waves; the R tiles of the partial wave are cut into
// S parts of their nkb K chunks, part c % S of tile W G + c / S going to CTA c < R S.  Valid tile t is
// n tile t % n_ntiles, row tile (t / n_ntiles) % nv, member t / (n_ntiles nv).
struct TailSched {
  int nv, W, R, S;
};
__device__ __forceinline__ TailSched tail_sched(const Args &p, int G, int nkb) {
  TailSched s;
  s.nv = min(p.meta[META_NPAD] / BM, p.n_rowtiles);
  const int Tv = p.n_ntiles * s.nv * p.n_members;
  s.W = Tv / G;
  s.R = Tv - s.W * G;
  s.S = s.R ? min(G / s.R, nkb) : 0;
  return s;
}
// the same waves, the R partial-wave tiles cut into S = NT / nsub_w column strips when R S <= G, else into
// two strips of NT / 2 columns (whole nsub_w-row boxes) when 2 R <= G, else not cut (S = 1)
__device__ __forceinline__ TailSched tail_sched_n(const Args &p, int G, int NTc) {
  TailSched s;
  s.nv = min(p.meta[META_NPAD] / BM, p.n_rowtiles);
  const int Tv = p.n_ntiles * s.nv * p.n_members;
  s.W = Tv / G;
  s.R = Tv - s.W * G;
  const int S = NTc / p.nsub_w;
  s.S = s.R * S <= G ? S : ((NTc % (2 * p.nsub_w) == 0 && 2 * s.R <= G) ? 2 : 1);
  return s;
}

// Shared memory of one CTA: the operand ring (1024-byte aligned for the 128-byte swizzle), then each
// epilogue warp's two output buffers (32 rows x 16 columns; hi and lo halves for the split), then the
// barriers.  The ring is as deep as the space allows (at most 6).
template <int NT, int EPI, int MODE, bool QUAD = false, int KB = BKB>
struct Smem {
  // halves per buffer (an fp32 piece of 32 rows x 8 columns fills one)
  static constexpr int OB = (EPI == EPI_F32 || EPI == EPI_ATOMIC) ? 1 : (MODE == MODE_SPLIT ? 2 : 1);
  static constexpr int WBUF = 1024;                                             // 32 rows x 32 bytes
  // output buffers per warp: two (one fills while the other's store reads), one where the ring needs
  // the space more (the split first layer: a fourth operand stage); the CELU' epilogue's buffers also
  // receive its aux pieces, loaded DCB pieces ahead (four for bf16 and fp8 operands; two for the split,
  // where four would cost it an operand stage: 106 -> 125 us for its second-layer backward)
  static constexpr int DCB = MODE == MODE_SPLIT ? 2 : 4;
  static constexpr int NBUF =
      (EPI == EPI_DCELU && !QUAD) ? DCB
                                  : ((MODE == MODE_SPLIT && EPI != EPI_F32 && EPI != EPI_ATOMIC && (EPI != EPI_DCELU || QUAD)) ? 1 : 2);
  static constexpr int OBYTES = OB ? EPI_WARPS * NBUF * OB * WBUF : 1024;
  static constexpr int FIXED = OBYTES + 1024 + 1024;
  static constexpr int AQ = QUAD ? 2 : 1;   // operand tiles per stage and side (hi, lo)
  static constexpr int FIT = (SMEM_LIMIT - FIXED) / (AQ * (BM * KB + NT * KB));
  static constexpr int STAGES = FIT > 6 ? 6 : FIT;
  uint8_t A[STAGES][AQ * BM * KB];
  uint8_t B[STAGES][AQ * NT * KB];
  uint8_t O[OBYTES];
  uint64_t full[STAGES], empty[STAGES], acc_full[2], acc_empty[2], fin, aux_bar[EPI_WARPS][4];
  uint32_t tmem_base;
  int abort_flag;
};

template <int NT, int EPI, int MODE, bool QUAD = false, int KB = BKB>
constexpr size_t smem_bytes() {
  return sizeof(Smem<NT, EPI, MODE, QUAD, KB>) + 1024;
}

// e^(z / alpha) as a power of two on the special-function unit (ex2.approx.ftz; z <= 0 where it is used, so
// the result lies in [0, 1] and results below the normal range flush to zero)
constexpr float CELU_EXP2 = CELU_INV_ALPHA * 1.4426950408889634f;   // log2(e) / alpha
__device__ __forceinline__ float exp_celu(float z) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(z * CELU_EXP2));
  return y;
}
__device__ __forceinline__ float celu_f(float z) { return z > 0.f ? z : CELU_ALPHA * (exp_celu(z) - 1.f); }
__device__ __forceinline__ float dcelu_h(float h) { return h > 0.f ? 1.f : 1.f + h * CELU_INV_ALPHA; }
__device__ __forceinline__ void epi_sync() { asm volatile("bar.sync 1, %0;" ::"n"(32 * EPI_WARPS) : "memory"); }
// OR of a predicate over the epilogue threads (named barrier 1): keeps their control flow uniform
__device__ __forceinline__ bool epi_any(bool pred) {
  uint32_t r;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\t"
      "setp.ne.u32 p, %1, 0;\n\t"
      "bar.red.or.pred q, 1, %2, p;\n\t"
      "selp.u32 %0, 1, 0, q;\n\t}\n"
      : "=r"(r)
      : "r"((uint32_t)pred), "n"(32 * EPI_WARPS)
      : "memory");
  return r != 0;
}

// tile t of the flattened grid -> (n tile, row tile, member); false when the row tile is padding.
// MODE_WG: (i tile, o tile, chunk, group): rt = o tile, m = member, e = element, r0 / nrows = its rows.
template <int MODE>
__device__ __forceinline__ bool tile_coords(const Args &p, int t, int &nt, int &rt, int &m, int &e, int &r0,
                                            int &nrows) {
  nt = t % p.n_ntiles;
  int rest = t / p.n_ntiles;
  rt = rest % p.n_rowtiles;
  rest /= p.n_rowtiles;
  if (MODE == MODE_WG) {
    const int chunk = rest % p.n_chunks, g = rest / p.n_chunks;
    m = g / NE;
    e = g - m * NE;
    const int s0 = p.seg[e], s1 = p.seg[e + 1];
    r0 = s0 + chunk * p.kchunk;
    nrows = min(p.kchunk, s1 - r0);
    return nrows > 0;
  }
  m = rest;
  e = p.tile_elem[rt];
  r0 = 0;
  nrows = 0;
  return e >= 0;
}

// Persistent: one CTA per SM walks tiles t = blockIdx.x, + gridDim.x, ...  Two TMEM accumulators
// (columns [0, 256) and [256, 512)) let the epilogue drain tile i while the MMAs of tile i+1 run.
// Each epilogue warp drains its own 32-row x 16-column pieces of a tile independently (no block-wide
// barrier): it converts them into one of its two shared-memory buffers and its lane 0 stores the
// piece with TMA while the warp fills the other buffer.  EPI_DCELU's aux piece is loaded by TMA into
// the buffer ahead of use and overwritten in place by the result.
template <int NT, int EPI, int MODE, bool QUAD = false, int KB = BKB>
__global__ void __launch_bounds__(THREADS, 1)
    k_umma(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
           const __grid_constant__ CUtensorMap tmA_lo, const __grid_constant__ CUtensorMap tmB_lo,
           const __grid_constant__ CUtensorMap tmO, const __grid_constant__ CUtensorMap tmO_lo,
           const __grid_constant__ CUtensorMap tmX, const __grid_constant__ CUtensorMap tmX_lo,
           const __grid_constant__ CUtensorMap tmBs, const __grid_constant__ CUtensorMap tmBs_lo, Args p) {
  static_assert(NT % 16 == 0 && NT >= 16 && NT <= 256, "UMMA N for M = 128");
  static_assert(!QUAD || MODE == MODE_SPLIT, "four-tile stages are a form of the split");
  static_assert(KB == BKB || QUAD, "64-byte rows only with four-tile stages");
  using SM = Smem<NT, EPI, MODE, QUAD, KB>;
  static_assert(SM::STAGES >= 2 && sizeof(SM) + 1024 <= SMEM_LIMIT, "shared memory budget");
  constexpr bool SPLIT = MODE == MODE_SPLIT, F8 = MODE == MODE_F8;
  constexpr int STAGES = SM::STAGES;
  constexpr int BK = F8 ? KB : KB / 2;   // K elements per stage
  extern __shared__ uint8_t smem_raw[];
  SM &S = *reinterpret_cast<SM *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  constexpr bool WG = MODE == MODE_WG;
  static_assert(!WG || (NT % 64 == 0 && KB == BKB), "MN-major operands: 64-feature boxes of 64 rows");
  const int nkb_fixed = (SPLIT && !QUAD) ? 3 * ((p.K + BK - 1) / BK) : (p.K + BK - 1) / BK;
  const int T = p.n_ntiles * p.n_rowtiles * p.n_members;
  volatile int *abort_flag = &S.abort_flag;
  // the work items of this CTA, in the same order for all three roles: tiles with their K chunk range
  // [kb0, kb1) (all of K but for tail parts) and whether the fp32 tile is added atomically
  const bool TS = EPI == EPI_F32 && p.tail_split;
  const bool TN = EPI != EPI_F32 && EPI != EPI_ATOMIC && EPI != EPI_L3 && !WG && p.tail_nsplit;
  TailSched ts{0, 0, 0, 0};
  if (TS) ts = tail_sched(p, (int)gridDim.x, nkb_fixed);
  if (TN) ts = tail_sched_n(p, (int)gridDim.x, NT);
  struct Item {
    int nt, rt, m, e, r0, nrows, kb0, kb1;
    bool atomic;
    int c0, cw;   // the item's columns of its tile: [c0, c0 + cw)
  };
  // 0: no more items, 1: skip (padding tile), 2: item
  auto item = [&](int it, Item &w) -> int {
    w.kb0 = 0;
    w.kb1 = -1;   // the tile's own count (nkb_fixed, or the WG chunk's)
    w.atomic = false;
    w.r0 = w.nrows = 0;
    w.c0 = 0;
    w.cw = NT;
    if (!TS && !TN) {
      const int t = (int)blockIdx.x + it * (int)gridDim.x;
      if (t >= T) return 0;
      return tile_coords<MODE>(p, t, w.nt, w.rt, w.m, w.e, w.r0, w.nrows) ? 2 : 1;
    }
    int t;
    if (it < ts.W) {
      t = (int)blockIdx.x + it * (int)gridDim.x;
    } else if (it == ts.W && (int)blockIdx.x < ts.R * ts.S) {
      const int part = (int)blockIdx.x % ts.S;
      t = ts.W * (int)gridDim.x + (int)blockIdx.x / ts.S;
      if (TS) {   // a K range, added atomically
        w.kb0 = part * nkb_fixed / ts.S;
        w.kb1 = (part + 1) * nkb_fixed / ts.S;
        w.atomic = true;
      } else if (ts.S > 1) {   // a column strip
        w.cw = NT / ts.S;
        w.c0 = part * w.cw;
      }
    } else {
      return 0;
    }
    w.nt = t % p.n_ntiles;
    const int rest = t / p.n_ntiles;
    w.rt = rest % ts.nv;
    w.m = rest / ts.nv;
    w.e = p.tile_elem[w.rt];
    return w.e >= 0 ? 2 : 1;
  };

  if (warp == 0 && lane == 0) {
    for (int s = 0; s < STAGES; s++) {
      mbar_init(&S.full[s], 1);
      mbar_init(&S.empty[s], 1);
    }
    for (int a = 0; a < 2; a++) {
      mbar_init(&S.acc_full[a], 1);
      mbar_init(&S.acc_empty[a], EPI_WARPS);   // one arrival per epilogue warp
      for (int w = 0; w < EPI_WARPS; w++) mbar_init(&S.aux_bar[w][a], 1), mbar_init(&S.aux_bar[w][2 + a], 1);
    }
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
    if (lane == 0) {  // ---- TMA producer: one continuous stage ring across this CTA's tiles
      long long g = 0, issued = 0;
      for (int it = 0; !*abort_flag; it++) {
        Item w;
        const int got = item(it, w);
        if (got == 0) break;
        if (got == 1) continue;
        const int nt = w.nt, rt = w.rt, m = w.m, e = w.e, r0 = w.r0, nrows = w.nrows;
        const int a_mid = p.a_by_member ? m : 0;
        const int b_grp = p.b_by_member ? m * NE + e : e;
        const int nkb_seg = WG ? (nrows + BK - 1) / BK : (p.K + BK - 1) / BK;
        const int nkb = w.kb1 >= 0 ? w.kb1 : (WG ? 2 * nkb_seg : nkb_fixed);
        for (int kb = w.kb0; kb < nkb; kb++, g++) {
          const int s = (int)(g % STAGES);
          if (g >= STAGES && !mbar_wait(&S.empty[s], (uint32_t)(((g / STAGES) - 1) & 1))) {
            *abort_flag = 1;
            break;
          }
          const bool strip = w.cw < NT;   // B rows nt NT + c0 .. + cw through the strip maps (nsub_w-row boxes)
          const CUtensorMap *mb = strip ? &tmBs : &tmB, *mb_lo = strip ? &tmBs_lo : &tmB_lo;
          const int by = nt * NT + w.c0;
          // the B rows of this item into dst: one box, or cw / nsub_w strip boxes one after another
          auto load_b = [&](uint8_t *dst, const CUtensorMap *map, int kc) {
            if (!strip) {
              tma_load_3d(dst, map, &S.full[s], kc, by, b_grp);
              return;
            }
            for (int h = 0; h < w.cw; h += p.nsub_w) tma_load_3d(dst + h * KB, map, &S.full[s], kc, by + h, b_grp);
          };
          mbar_expect_tx(&S.full[s], (uint32_t)(SM::AQ * (BM + w.cw) * KB));
          if (QUAD) {   // hi and lo of both operands for one K chunk
            tma_load_3d(S.A[s], &tmA, &S.full[s], kb * BK, a_mid, rt * BM);
            tma_load_3d(S.A[s] + BM * KB, &tmA_lo, &S.full[s], kb * BK, a_mid, rt * BM);
            load_b(S.B[s], mb, kb * BK);
            load_b(S.B[s] + NT * KB, mb_lo, kb * BK);
          } else if (WG) {   // term 0 (A, B), then term 1 (A_lo, B_lo): BK rows x 64 features per box
            const int term = kb / nkb_seg, y = r0 + (kb - term * nkb_seg) * BK;
            const CUtensorMap *ma = term ? &tmA_lo : &tmA, *mbw = term ? &tmB_lo : &tmB;
#pragma unroll
            for (int j = 0; j < BM / 64; j++) tma_load_3d(S.A[s] + j * BK * 128, ma, &S.full[s], rt * BM + 64 * j, m, y);
#pragma unroll
            for (int j = 0; j < NT / 64; j++)
              tma_load_3d(S.B[s] + j * BK * 128, mbw, &S.full[s], nt * NT + 64 * j, p.b_shared ? 0 : m, y);
          } else {
            const int seg = SPLIT ? kb / nkb_seg : 0, kk = SPLIT ? kb - seg * nkb_seg : kb;
            tma_load_3d(S.A[s], seg == 2 ? &tmA_lo : &tmA, &S.full[s], kk * BK, a_mid, rt * BM);
            load_b(S.B[s], seg == 1 ? mb_lo : mb, kk * BK);
          }
          issued = g + 1;
        }
      }
      // drain: every issued load must land before the CTA can exit
      for (long long q = (issued > STAGES ? issued - STAGES : 0); q < issued; q++)
        if (!mbar_wait(&S.full[q % STAGES], (uint32_t)((q / STAGES) & 1))) *abort_flag = 1;
    }
  } else if (warp == 1) {
    if (lane == 0) {  // ---- MMA issuer
      const uint32_t idesc = F8 ? idesc_e4m3(BM, NT) : (WG ? idesc_bf16_mn(BM, NT) : idesc_bf16(BM, NT));
      long long g = 0;
      int cnt = 0;
      for (int it = 0; !*abort_flag; it++) {
        Item w;
        const int got = item(it, w);
        if (got == 0) break;
        if (got == 1) continue;
        const int kb0 = w.kb0;
        const int nkb = w.kb1 >= 0 ? w.kb1 : (WG ? 2 * ((w.nrows + BK - 1) / BK) : nkb_fixed);
        const uint32_t id = w.cw == NT ? idesc : (F8 ? idesc_e4m3(BM, w.cw) : idesc_bf16(BM, w.cw));
        const int a = cnt & 1;
        if (cnt >= 2 && !mbar_wait(&S.acc_empty[a], (uint32_t)(((cnt >> 1) - 1) & 1))) {
          *abort_flag = 1;
          break;
        }
        fence_after();
        const uint32_t d = tmem + (uint32_t)(a * TMEM_COLS);
        for (int kb = kb0; kb < nkb; kb++, g++) {
          const uint32_t acc0 = kb != kb0 ? 1u : 0u;   // the item's first K step starts the accumulator
          const int s = (int)(g % STAGES);
          if (!mbar_wait(&S.full[s], (uint32_t)((g / STAGES) & 1))) {
            *abort_flag = 1;
            break;
          }
          fence_after();
          const uint32_t a0 = smem_u32(S.A[s]), b0 = smem_u32(S.B[s]);
#pragma unroll
          for (int k = 0; k < KB / 32; k++) {
            const uint32_t acc = (acc0 | (uint32_t)k) != 0 ? 1u : 0u;
            if (QUAD) {   // hi hi + hi lo + lo hi of this K step
              const uint64_t ah = sdesc<KB>(a0 + 32 * k), al = sdesc<KB>(a0 + BM * KB + 32 * k);
              const uint64_t bh = sdesc<KB>(b0 + 32 * k), bl = sdesc<KB>(b0 + NT * KB + 32 * k);
              mma_bf16(d, ah, bh, id, acc);
              mma_bf16(d, ah, bl, id, 1u);
              mma_bf16(d, al, bh, id, 1u);
            } else if (WG) {   // 16 K rows of 128 bytes per step
              mma_bf16(d, sdesc_mn_sw128(a0 + 2048 * k, BK * 128), sdesc_mn_sw128(b0 + 2048 * k, BK * 128), id, acc);
            } else if (F8)
              mma_f8(d, sdesc_sw128(a0 + 32 * k), sdesc_sw128(b0 + 32 * k), id, acc);
            else
              mma_bf16(d, sdesc<KB>(a0 + 32 * k), sdesc<KB>(b0 + 32 * k), id, acc);
          }
          mma_commit(&S.empty[s]);
        }
        if (*abort_flag) break;
        mma_commit(&S.acc_full[a]);  // accumulator a complete once these MMAs finish
        cnt++;
      }
      // every MMA issued above must be complete before TMEM can be released
      mma_commit(&S.fin);
      if (!mbar_wait(&S.fin, 0)) *abort_flag = 1;
    }
  } else {  // ---- epilogue warps 2 .. 2 + EPI_WARPS - 1
    const int q = warp & 3;                 // TMEM lane quarter this warp may read
    const int part = (warp - 2) >> 2;       // which of the quarter's four warps: chunks part, part + 4, ...
    const int r = q * 32 + lane;
    const int ew = warp - 2;                // epilogue warp index
    constexpr int PB = F8 ? 16 * 32 : 32 * 32;   // bytes of one 32 x 16 piece
    uint8_t *wb = S.O + (size_t)ew * SM::NBUF * SM::OB * SM::WBUF;   // this warp's buffers
    uint32_t aux_phase = 0u;                // bit b: the parity of buffer b's next aux load
    unsigned aux_out = 0;                   // lane 0: buffers with an aux load not yet consumed
    long long gk = 0;                       // pieces drained by this warp (buffer gk & 1)
    int cnt = 0;
    int nt_cur = 0;                         // n tile of the tile being drained (aux y coordinate, x_y == 2)
    // lane 0: aux piece (columns col.. col + 15 of tile (rt, m)) into buffer b
    auto load_aux = [&](int b, int col, int rt, int m) {
      uint8_t *ob = wb + (size_t)b * SM::OB * SM::WBUF;
      mbar_expect_tx(&S.aux_bar[ew][b], (uint32_t)(SPLIT ? 2 * PB : PB));
      const int y = p.x_y == 1 ? m : p.x_y == 2 ? nt_cur : 0;
      tma_load_3d(ob, &tmX, &S.aux_bar[ew][b], col, y, rt * BM + q * 32);
      if (SPLIT) tma_load_3d(ob + SM::WBUF, &tmX_lo, &S.aux_bar[ew][b], col, y, rt * BM + q * 32);
      aux_out |= 1u << b;
    };
    for (int it = 0;; it++) {
      Item w;
      const int got = item(it, w);
      if (got == 0) break;
      if (got == 1) continue;
      const int nt = w.nt, rt = w.rt, m = w.m, e = w.e;
      const int a = cnt & 1;
      const int n0 = nt * NT;
      const int ncols = min(NT, p.N - n0);
      nt_cur = nt;
      // the first aux pieces of the tile, one per buffer (the loads stay NBUF pieces ahead), travel while
      // its MMAs run
      const int cend = min(ncols, w.c0 + w.cw);   // the item's columns (tile coordinates)
      if (EPI == EPI_DCELU && lane == 0 && w.c0 + 16 * part < cend) {
        if (gk >= 1) bulk_wait_read0();   // the stores that last read the buffers
#pragma unroll
        for (int i = 0; i < SM::NBUF; i++)
          if (w.c0 + 16 * part + 64 * i < cend) load_aux((int)((gk + i) % SM::NBUF), w.c0 + 16 * part + 64 * i, rt, m);
      }
      const float *bias = p.bias + e * p.bias_estride + m * p.bias_mstride + n0;
      // the bias of this warp's pieces, read while the MMAs run: lane j holds column j of each piece (one
      // value per piece, broadcast by shuffles below), so no load waits inside the drain
      constexpr int NPB = (NT + 63) / 64;
      float pre[NPB];
      if (EPI == EPI_BIAS_CELU) {
#pragma unroll
        for (int i = 0; i < NPB; i++) {
          const int c = w.c0 + 16 * part + 64 * i;
          pre[i] = c < cend ? __ldg(bias + c + (lane & 15)) : 0.f;
        }
      }
      bool ok = mbar_wait(&S.acc_full[a], (uint32_t)((cnt >> 1) & 1));
      fence_after();
      if (!__all_sync(0xffffffffu, ok)) {
        *abort_flag = 1;
        break;
      }
      const long long row = (long long)rt * BM + r;
      const uint32_t tbase = tmem + (uint32_t)(a * TMEM_COLS) + ((uint32_t)(q * 32) << 16);
      float ysum = 0.f;
      float sc = 1.f;   // dequantisation of the fp8 product
      if (F8) sc = p.a_scale * p.b_scale[(p.b_scale_by == 1 ? m : p.b_scale_by == 2 ? nt : 0) * NE + e];
      const float *w4 = p.w4 + e * p.w4_estride + m * p.w4_mstride + n0;
      const int oy = p.o_y == 1 ? m : p.o_y == 2 ? nt : 0;
      bool abort_now = false;
#pragma unroll 1
      for (int c = w.c0 + 16 * part; c < w.c0 + w.cw; c += 64) {
        float pb = 0.f;   // this piece's prefetched bias (lane j: column j)
        if (EPI == EPI_BIAS_CELU) {
          pb = pre[0];
#pragma unroll
          for (int i = 0; i + 1 < NPB; i++) pre[i] = pre[i + 1];
        }
        float v[16];
        tmem_ld16(tbase + (c - w.c0), v);
        if (c >= ncols) continue;  // warp-uniform; ncols is a multiple of 16 in every use
        if (EPI == EPI_ATOMIC && rt * BM + q * 32 >= p.O) continue;   // rows beyond dW (warp-uniform)
        if (EPI == EPI_ATOMIC || EPI == EPI_F32) {
          // 32-row x 8-column fp32 pieces through this warp's two buffers, by TMA: the weight-gradient tile
          // (rows o of dW[m][e]) added into dW; the input gradient stored, or for a K part of a tail tile
          // added into the tile zeroed beforehand
          const float k = EPI == EPI_F32 ? sc * p.scale : 1.f;
#pragma unroll
          for (int hh = 0; hh < 2; hh++) {
            uint8_t *ob = wb + (size_t)(gk & 1) * SM::WBUF;
            if (lane == 0 && gk >= 2) bulk_wait_read1();   // the operation that last read this buffer
            __syncwarp();
            float4 *d4 = reinterpret_cast<float4 *>(ob + lane * 32);
            d4[0] = make_float4(v[8 * hh] * k, v[8 * hh + 1] * k, v[8 * hh + 2] * k, v[8 * hh + 3] * k);
            d4[1] = make_float4(v[8 * hh + 4] * k, v[8 * hh + 5] * k, v[8 * hh + 6] * k, v[8 * hh + 7] * k);
            fence_proxy_async();
            __syncwarp();
            if (lane == 0) {
              if (EPI == EPI_ATOMIC)
                tma_reduce_add_3d(&tmO, ob, n0 + c + 8 * hh, rt * BM + q * 32, m * NE + e);
              else if (w.atomic)
                tma_reduce_add_3d(&tmO, ob, n0 + c + 8 * hh, 0, rt * BM + q * 32);
              else
                tma_store_3d(&tmO, ob, n0 + c + 8 * hh, 0, rt * BM + q * 32);
              bulk_commit();
            }
            gk++;
          }
          continue;
        }
        const int b = (int)(gk % SM::NBUF);
        uint8_t *ob = wb + (size_t)b * SM::OB * SM::WBUF;
        if (EPI == EPI_DCELU) {
          const bool got = mbar_wait(&S.aux_bar[ew][b], (aux_phase >> b) & 1u);
          aux_phase ^= 1u << b;
          if (lane == 0) aux_out &= ~(1u << b);
          if (!__all_sync(0xffffffffu, got)) {
            abort_now = true;
            break;
          }
        } else {
          if (lane == 0 && SM::NBUF == 2 && gk >= 2) bulk_wait_read1();
          if (lane == 0 && SM::NBUF == 1 && gk >= 1) bulk_wait_read0();
          __syncwarp();
        }
        if (F8)
#pragma unroll
          for (int j = 0; j < 16; j++) v[j] *= sc;
        float f[16];
        if (EPI == EPI_PLAIN) {
#pragma unroll
          for (int j = 0; j < 16; j++) f[j] = v[j];
        } else if (EPI == EPI_BIAS_CELU) {
#pragma unroll
          for (int j = 0; j < 16; j++) f[j] = celu_f(v[j] + __shfl_sync(0xffffffffu, pb, j));
        } else if (EPI == EPI_L3) {
#pragma unroll
          for (int j = 0; j < 16; j += 4) {
            const float4 bb = __ldg(reinterpret_cast<const float4 *>(bias + c + j));
            const float4 ww = __ldg(reinterpret_cast<const float4 *>(w4 + c + j));
            const float zb[4] = {bb.x, bb.y, bb.z, bb.w}, wv[4] = {ww.x, ww.y, ww.z, ww.w};
#pragma unroll
            for (int u = 0; u < 4; u++) {
              const float z = v[j + u] + zb[u];
              const float ez = exp_celu(fminf(z, 0.f));
              ysum += (z > 0.f ? z : CELU_ALPHA * (ez - 1.f)) * wv[u];
              f[j + u] = p.scale * wv[u] * (z > 0.f ? 1.f : ez);
            }
          }
        } else {  // EPI_DCELU: aux h of this row and columns, from the buffer
          float hv[16];
          if (F8) {
            alignas(16) __nv_fp8x2_storage_t hq[8];
            *reinterpret_cast<uint4 *>(hq) = *reinterpret_cast<const uint4 *>(ob + lane * 16);
#pragma unroll
            for (int j = 0; j < 8; j++) {
              const float2 h2 = __half22float2(__half2(__nv_cvt_fp8x2_to_halfraw2(hq[j], __NV_E4M3)));
              hv[2 * j] = h2.x * p.aux_scale;
              hv[2 * j + 1] = h2.y * p.aux_scale;
            }
          } else {
            alignas(16) __nv_bfloat16 hb[16];
            *reinterpret_cast<uint4 *>(hb) = *reinterpret_cast<const uint4 *>(ob + lane * 32);
            *reinterpret_cast<uint4 *>(hb + 8) = *reinterpret_cast<const uint4 *>(ob + lane * 32 + 16);
#pragma unroll
            for (int j = 0; j < 16; j++) hv[j] = __bfloat162float(hb[j]);
            if (SPLIT) {
              *reinterpret_cast<uint4 *>(hb) = *reinterpret_cast<const uint4 *>(ob + SM::WBUF + lane * 32);
              *reinterpret_cast<uint4 *>(hb + 8) = *reinterpret_cast<const uint4 *>(ob + SM::WBUF + lane * 32 + 16);
#pragma unroll
              for (int j = 0; j < 16; j++) hv[j] += __bfloat162float(hb[j]);
            }
          }
#pragma unroll
          for (int j = 0; j < 16; j++) f[j] = v[j] * dcelu_h(hv[j]);
        }
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
          const int x = p.o_xm * m + c;
          tma_store_3d(&tmO, ob, x, oy, rt * BM + q * 32);
          if (SPLIT) tma_store_3d(&tmO_lo, ob + SM::WBUF, x, oy, rt * BM + q * 32);
          bulk_commit();
          if (EPI == EPI_DCELU && c + 64 * SM::NBUF < cend) {   // the piece NBUF on into this buffer, once read
            bulk_wait_read0();
            load_aux(b, c + 64 * SM::NBUF, rt, m);
          }
        }
        gk++;
      }
      if (abort_now) {
        *abort_flag = 1;
        break;
      }
      if (EPI == EPI_L3) p.ypart[(row * p.M + m) * 4 + part] = ysum;
      // accumulator a may be overwritten once every epilogue warp has read it
      fence_before();
      __syncwarp();
      if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&S.acc_empty[a])) : "memory");
      cnt++;
    }
    if (lane == 0) {
      // nothing may still read or write this warp's buffers when the CTA exits
      bulk_wait_all();
      for (int b = 0; b < SM::NBUF; b++)
        if ((aux_out >> b) & 1u)
          if (!mbar_wait(&S.aux_bar[ew][b], (aux_phase >> b) & 1u)) *abort_flag = 1;
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
