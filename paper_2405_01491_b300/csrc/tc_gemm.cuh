// tcgen05 (5th-generation tensor core) GEMM for the per-element networks, sm_103a.
//
// One CTA computes a 128 x NT tile C = A B^T of a "TN" product (both operands K-contiguous):
//   warp 0 (one lane)  TMA producer: 128x64 A and NTx64 B bf16 tiles, 128-byte swizzle, STAGES-deep
//                      ring guarded by full/empty mbarriers
//   warp 1 (one lane)  MMA issuer: 4 x tcgen05.mma (K = 16 each) per stage, accumulator in TMEM
//                      (128 lanes x NT fp32 columns); tcgen05.commit frees the stage
//   warps 2-5          epilogue: tcgen05.ld 32 lanes x 16 columns at a time (warp w reads TMEM lane
//                      quarter w % 4), fused bias/CELU, CELU', output-layer dot, store
// Every mbarrier wait is bounded; on timeout the CTA posts FNN_E_TIMEOUT, drains what it issued,
// frees its TMEM and returns.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>

#include "fnn_internal.cuh"

namespace fnn {
namespace tc {

constexpr int STAGES = 4;
constexpr int BM = 128;         // rows per tile (UMMA M)
constexpr int BK = 64;          // K per stage: 64 bf16 = one 128-byte swizzle row
constexpr int TMEM_COLS = 256;  // accumulator columns allocated (NT <= 256)
constexpr int THREADS = 192;
constexpr long long WAIT_LIMIT = 2000000000LL;  // clock64 cycles (about a second) before a wait gives up

enum { EPI_BIAS_CELU = 0, EPI_L3 = 1, EPI_DCELU = 2, EPI_F32 = 3 };

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
// arrive on an mbarrier once every previously issued tcgen05.mma of this thread has completed
__device__ __forceinline__ void mma_commit(uint64_t *bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

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

// Instruction descriptor, kind::f16: fp32 accumulator [4,6) = 1, A and B bf16 [7,10) = [10,13) = 1,
// both K-major (bits 15, 16 = 0), N >> 3 at [17,23), M >> 4 at [24,29).
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// ---------------------------------------------------------------------------------- kernel
struct Args {
  int K;                       // reduction length
  int N;                       // valid output columns of the whole product
  int a_by_member;             // A's middle coordinate = member (else 0)
  int b_by_member;             // B's group coordinate = member * 7 + element (else element)
  const int32_t *tile_elem;    // element of each 128-row tile (-1: skip)
  void *out;                   // bf16 (or fp32 for EPI_F32) [rows][ldo]
  long long ldo, o_mstride;
  const float *bias;
  long long bias_estride, bias_mstride;
  const __nv_bfloat16 *aux;    // h of the previous layer (EPI_DCELU)
  long long ldaux, aux_mstride;
  const float *w4;             // output layer (EPI_L3)
  long long w4_estride, w4_mstride;
  float *ypart;                // [rows][M][4] (EPI_L3, column 0)
  int M;
  float scale;
  DevStatus *st;
};

template <int NT>
struct Smem {
  __nv_bfloat16 A[STAGES][BM * BK];
  __nv_bfloat16 B[STAGES][NT * BK];
  uint64_t full[STAGES], empty[STAGES], done;
  uint32_t tmem_base;
  int abort_flag;
};

template <int NT>
constexpr size_t smem_bytes() {
  return sizeof(Smem<NT>) + 1024;
}

__device__ __forceinline__ float celu_f(float z) { return z > 0.f ? z : CELU_ALPHA * (__expf(z / CELU_ALPHA) - 1.f); }
__device__ __forceinline__ float dcelu_h(float h) { return h > 0.f ? 1.f : 1.f + h / CELU_ALPHA; }

template <int NT, int EPI>
__global__ void __launch_bounds__(THREADS, 1)
    k_umma(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, Args p) {
  static_assert(NT % 16 == 0 && NT >= 16 && NT <= 256, "UMMA N for M = 128");
  const int e = p.tile_elem[blockIdx.y];
  if (e < 0) return;
  extern __shared__ uint8_t smem_raw[];
  Smem<NT> &S = *reinterpret_cast<Smem<NT> *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m = blockIdx.z;
  const int row0 = blockIdx.y * BM, n0 = blockIdx.x * NT;
  const int nkb = (p.K + BK - 1) / BK;

  if (warp == 0 && lane == 0) {
    for (int s = 0; s < STAGES; s++) {
      mbar_init(&S.full[s], 1);
      mbar_init(&S.empty[s], 1);
    }
    mbar_init(&S.done, 1);
    S.abort_flag = 0;
    fence_barrier_init();
  }
  if (warp == 1) {
    tmem_alloc(&S.tmem_base, TMEM_COLS);
    tmem_relinquish();
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = S.tmem_base;

  if (warp == 0) {
    if (lane == 0) {  // ---- TMA producer
      const int a_mid = p.a_by_member ? m : 0;
      const int b_grp = p.b_by_member ? m * NE + e : e;
      int issued = 0;
      for (int kb = 0; kb < nkb; kb++) {
        const int s = kb % STAGES;
        if (kb >= STAGES && !mbar_wait(&S.empty[s], ((kb / STAGES) - 1) & 1)) {
          S.abort_flag = 1;
          break;
        }
        if (*(volatile int *)&S.abort_flag) break;
        mbar_expect_tx(&S.full[s], (uint32_t)((BM + NT) * BK * 2));
        tma_load_3d(S.A[s], &tmA, &S.full[s], kb * BK, a_mid, row0);
        tma_load_3d(S.B[s], &tmB, &S.full[s], kb * BK, n0, b_grp);
        issued = kb + 1;
      }
      // drain: every issued load must land before the CTA can exit
      for (int kb = (issued > STAGES ? issued - STAGES : 0); kb < issued; kb++)
        if (!mbar_wait(&S.full[kb % STAGES], (kb / STAGES) & 1)) S.abort_flag = 1;
    }
  } else if (warp == 1) {
    if (lane == 0) {  // ---- MMA issuer
      const uint32_t idesc = idesc_bf16(BM, NT);
      for (int kb = 0; kb < nkb; kb++) {
        const int s = kb % STAGES;
        if (!mbar_wait(&S.full[s], (kb / STAGES) & 1)) {
          S.abort_flag = 1;
          break;
        }
        if (*(volatile int *)&S.abort_flag) break;
        fence_after();
        const uint32_t a0 = smem_u32(S.A[s]), b0 = smem_u32(S.B[s]);
#pragma unroll
        for (int k = 0; k < BK / 16; k++)
          mma_bf16(tmem, sdesc_sw128(a0 + 32 * k), sdesc_sw128(b0 + 32 * k), idesc, (kb | k) != 0);
        mma_commit(&S.empty[s]);
      }
      mma_commit(&S.done);  // arrives once every MMA issued above has completed
    }
  } else {  // ---- epilogue warps 2..5
    const bool ok = __all_sync(0xffffffffu, mbar_wait(&S.done, 0));
    fence_after();
    if (!ok) S.abort_flag = 1;
    const int q = warp & 3;
    const int r = q * 32 + lane;
    const long long row = (long long)row0 + r;
    const uint32_t tbase = tmem + ((uint32_t)(q * 32) << 16);
    float ysum = 0.f;
    if (ok) {
#pragma unroll 1
      for (int c = 0; c < NT; c += 16) {
        float v[16];
        tmem_ld16(tbase + c, v);
        const int n = n0 + c;
        if (n >= p.N) continue;  // N is a multiple of 16 in every use
        if (EPI == EPI_F32) {
          float *o = reinterpret_cast<float *>(p.out) + row * p.ldo + m * p.o_mstride + n;
#pragma unroll
          for (int j = 0; j < 16; j += 4)
            *reinterpret_cast<float4 *>(o + j) =
                make_float4(v[j] * p.scale, v[j + 1] * p.scale, v[j + 2] * p.scale, v[j + 3] * p.scale);
        } else {
          __nv_bfloat16 *o = reinterpret_cast<__nv_bfloat16 *>(p.out) + row * p.ldo + m * p.o_mstride + n;
          alignas(16) __nv_bfloat16 ob[16];
          if (EPI == EPI_BIAS_CELU) {
            const float *b = p.bias + e * p.bias_estride + m * p.bias_mstride + n;
#pragma unroll
            for (int j = 0; j < 16; j++) ob[j] = __float2bfloat16(celu_f(v[j] + b[j]));
          } else if (EPI == EPI_L3) {
            const float *b = p.bias + e * p.bias_estride + m * p.bias_mstride + n;
            const float *w = p.w4 + e * p.w4_estride + m * p.w4_mstride + n;
#pragma unroll
            for (int j = 0; j < 16; j++) {
              float z = v[j] + b[j];
              ysum += celu_f(z) * w[j];
              ob[j] = __float2bfloat16(p.scale * w[j] * (z > 0.f ? 1.f : __expf(z / CELU_ALPHA)));
            }
          } else {  // EPI_DCELU
            const __nv_bfloat16 *h = p.aux + row * p.ldaux + m * p.aux_mstride + n;
            alignas(16) __nv_bfloat16 hb[16];
            *reinterpret_cast<uint4 *>(hb) = *reinterpret_cast<const uint4 *>(h);
            *reinterpret_cast<uint4 *>(hb + 8) = *reinterpret_cast<const uint4 *>(h + 8);
#pragma unroll
            for (int j = 0; j < 16; j++) ob[j] = __float2bfloat16(v[j] * dcelu_h(__bfloat162float(hb[j])));
          }
          *reinterpret_cast<uint4 *>(o) = *reinterpret_cast<const uint4 *>(ob);
          *reinterpret_cast<uint4 *>(o + 8) = *reinterpret_cast<const uint4 *>(ob + 8);
        }
      }
      if (EPI == EPI_L3) p.ypart[(row * p.M + m) * 4] = ysum;
    }
  }
  fence_before();
  __syncthreads();
  if (S.abort_flag && threadIdx.x == 0) post_status(p.st, FNN_E_TIMEOUT, blockIdx.y);
  if (warp == 1) {
    fence_after();
    tmem_dealloc(tmem, TMEM_COLS);
  }
}

}  // namespace tc
}  // namespace fnn
