// ANI atomic environment vectors and their adjoint (sections II.A, II.B, II.E; Appendix A).
//
// One warp per centre atom.  The warp stages its neighbour row into shared memory bucketed by
// element (two ballot passes: count per element, then scatter), keeping the entries within
// rc_rad (radial list) and the subset within rc_ang (angular list).
//
// Forward, radial: for each element segment, lane (h, k) = (lane / 16, lane % 16) sums shift k
// over every other neighbour; one shuffle joins the halves; 16 lanes write 64 contiguous bytes.
// Forward, angular: all unordered pairs j < k of the element-sorted angular list in batches of 32,
// enumerated block by block in slot order (element pair (a, b), a <= b).  Each lane evaluates one
// triplet (4 section powers, 8 radial Gaussians times the switch product) into a shared staging
// row; then lane (m, s) = (lane / 4, lane % 4) sums pow_s(t) * gauss_m(t) over the batch into a
// register that is stored (coalesced, 32 slots per pair) when the pair's block ends.
// Adjoint: same staging and enumeration; per triplet the lane reads its pair's 32 gradient slots
// from a padded shared row, chains the partials to dE/dd per neighbour in shared memory, then the
// warp scatters them to the forces (F_j -= g, F_i += g) and the virial -d (x) g.
#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include "fnn_internal.cuh"
#include "tc_gemm.cuh"

namespace fnn {

static constexpr unsigned FULL = 0xffffffffu;
constexpr int AEV_WARPS = 4, ADJ_WARPS = 4;
constexpr int AEV_FWD_BLOCKS = 8, AEV_ADJ_BLOCKS = 5;   // resident blocks per SM (shared memory)

// 2^x on the special-function unit (ex2.approx.ftz: about 2 ulp; arguments here are <= 0)
__device__ __forceinline__ float exp2f_fast(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// log2 on the special-function unit (lg2.approx.ftz: about 2 ulp; the arguments are switch values in
// [0, 1] and section bases above 0.1, and a zero switch value gives -inf, whose power of two is zero)
__device__ __forceinline__ float log2_fast(float x) {
  float y;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// reciprocal and square root on the special-function unit (rcp.approx / sqrt.approx: about 1 ulp; the
// arguments are normal numbers: distances above 0.5 A, the section base above 0.1, sin theta' above 0.3)
__device__ __forceinline__ float rcp_fast(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float sqrt_fast(float x) {
  float y;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// Two FP32 operations in one instruction (the packed add, multiply and fma of this architecture, each half
// rounded as its scalar form): the AEV kernels are bound by instruction issue, and their shift and section
// loops are pairs of independent streams of arithmetic
__device__ __forceinline__ float2 dup2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 exp2_2(float2 x) { return make_float2(exp2f_fast(x.x), exp2f_fast(x.y)); }
__device__ __forceinline__ float2 log2_2(float2 x) { return make_float2(log2_fast(x.x), log2_fast(x.y)); }
__device__ __forceinline__ float2 rcp_2(float2 x) { return make_float2(rcp_fast(x.x), rcp_fast(x.y)); }

// 16-byte copies global -> shared (cp.async, L2 only), their commit groups and waits
__device__ __forceinline__ void cp16(void *smem, const void *gmem) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((unsigned)__cvta_generic_to_shared(smem)),
               "l"(gmem)
               : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_wait1() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }
__device__ __forceinline__ void cp_wait0() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// per-warp staging of one centre atom's neighbours, bucketed by element, for the adjoint and the tangent
// (the switch values of radial entries are recomputed from r where used)
template <bool FULL>
struct NbrStageT {
  float4 rd[RAD_CAP];            // dx, dy, dz, r   (element-sorted, r < rc_rad)
  int rj[RAD_CAP];               // neighbour atom
  unsigned char re[RAD_CAP];     // element per radial entry
  unsigned char aidx[ANG_CAP];   // angular entry -> radial entry
  unsigned char ae[ANG_CAP];     // angular entry element
  float afc[ANG_CAP];            // angular switch fc(r; rc_ang)
  float adfc[ANG_CAP];           // its derivative
};
using NbrStage = NbrStageT<true>;
constexpr int SROW = 36;         // padded staging row: rows s (or m) start 4 banks apart

// The non-empty element-pair blocks of an atom's triplets in slot order, then one past the last:
// bt = {first slot, j0 | k0 << 8 | (a == b) << 16, count of element b, count of element a} with j0, k0 the
// angular-list starts of elements a and b, {slots, 0, 0, 0} past the last (a block of t triplets takes t
// rounded up to a multiple of four slots); bi = 1 / count of a (a == b) or of b, the divisor of the block's
// pair index; bq = slot block | t << 8
struct BlockTable {
  int4 bt[NPAIR + 1];
  float bi[NPAIR + 1];
  int bq[NPAIR + 1];
};

// The forward's staging of one centre atom: only what its sums read, in the form they read it
struct FwdNbr {
  float2 rr[RAD_CAP];            // r, log2 fc(r; rc_rad) - 2   (element-sorted, r < rc_rad; the 1/4 prefactor)
  float4 au[ANG_CAP];            // unit vector to the neighbour, r / 2   (element-sorted, r < rc_ang)
  float la[ANG_CAP];             // log2 fc(r; rc_ang) + 1/2: la_j + la_k = log2(2 fc_j fc_k)
};
struct FwdStage {
  FwdNbr nb;
  // per-triplet factors of one batch, triplet innermost so a consumer lane reads four at once:
  // 4 section powers and 8 Gaussians x switches
  alignas(16) float sf[NSZ][SROW];
  alignas(16) float sg[NSA][SROW];
  int sp[32];                    // slot block of a triplet that opens one
  BlockTable tb;
};
constexpr int GS_STRIDE = 36;
struct AdjStage {
  NbrStage nb;
  float gacc[RAD_CAP][3];        // dE/dd per radial entry
  double vacc[9];                // virial of the current structure (lane 0), flushed when it changes
  // the angular part of the atom's dE/dAEV row ([pair][m][s]), GS_STRIDE floats per pair: the lanes of a
  // batch read the rows of different pairs at the same offset, which then fall in different banks (with 32
  // floats per pair every lane's float4 hit the same four banks: 134.9 -> 129.9 us on the 23,558-atom box)
  alignas(16) float gs[NPAIR * GS_STRIDE];
};

struct StageArgs {
  int64_t cap;            // list capacity: entries at or beyond it were never written
  int sorted_upto;        // rows of at most this many entries are sorted by neighbour element
  const float4 *pos;
  const int32_t *row_ptr, *nbr;
  const char4 *shift;
  const uint8_t *elem;
  const int32_t *atom_mol;
  const MolGrid *grid;
};

// Stage atom i's neighbours; returns false when the atom has no structure, or (after posting
// FNN_E_CAPACITY) when a list overflows.  The per-element counts are kept one element per lane: on return
// lane q < NE holds the start of element q's radial (orr) and angular (oa) segment and their counts (cr,
// ca); lane NE holds the totals in orr and oa.  A row sorted by neighbour element (see PAIR_STRIDE) is
// staged in one pass, its radial and angular subsets in list order; any other row in two (count, then
// scatter, stable within an element).
template <bool FULL>
__device__ bool stage_neighbors(const StageArgs &A, const AevParams &P, int i, NbrStageT<FULL> &S, int &orr,
                                int &oa, int &cr, int &ca, DevStatus *st) {
  const int lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1u;
  const int mol = A.atom_mol[i];
  if (mol < 0) return false;   // atom outside every structure (already posted)
  const float4 pi = A.pos[i];
  const MolGrid &g = A.grid[mol];
  const int pbc = g.pbc;
  const float Lx = pbc ? g.Lx : 0.f, Ly = pbc ? g.Ly : 0.f, Lz = pbc ? g.Lz : 0.f;
  const int k0 = (int)min((int64_t)A.row_ptr[i], A.cap), k1 = (int)min((int64_t)A.row_ptr[i + 1], A.cap);
  // list entry k (< k1) of this lane: separation, distance, element and the two cutoff tests
  auto entry = [&](int k, int &j, float &dx, float &dy, float &dz, float &r, int &e, bool &vr, bool &va) {
    vr = va = false;
    e = 0;
    j = 0;
    dx = dy = dz = r = 0.f;
    if (k < k1) {
      j = A.nbr[k];
      const char4 sh = A.shift[k];
      const float4 pj = A.pos[j];
      dx = (pj.x - pi.x) + (float)sh.x * Lx;
      dy = (pj.y - pi.y) + (float)sh.y * Ly;
      dz = (pj.z - pi.z) + (float)sh.z * Lz;
      r = sqrt_fast(dx * dx + dy * dy + dz * dz);
      vr = r < P.rc_rad;
      va = r < P.rc_ang;
      e = A.elem[j];
    }
  };
  auto put = [&](int pr, int pa, int j, float dx, float dy, float dz, float r, int e) {
    S.rd[pr] = make_float4(dx, dy, dz, r);
    S.rj[pr] = j;
    S.re[pr] = (unsigned char)e;
    if (pa >= 0) {
      S.aidx[pa] = (unsigned char)pr;
      S.ae[pa] = (unsigned char)e;
      S.afc[pa] = switch_f(P, r, P.rc_ang, P.inv_rc_ang);
      S.adfc[pa] = switch_df(P, r, P.rc_ang, P.inv_rc_ang, P.pi_rc_ang);
    }
  };
  const bool sorted = k1 - k0 <= A.sorted_upto;
  cr = ca = 0;   // lane q < NE: entries of element q
  int nr = 0, na = 0;
  for (int kb = k0; kb < k1; kb += 32) {   // sorted rows: the only pass; others: counts
    int j, e;
    float dx, dy, dz, r;
    bool vr, va;
    entry(kb + lane, j, dx, dy, dz, r, e, vr, va);
    const unsigned mr = __ballot_sync(FULL, vr), ma = __ballot_sync(FULL, va);
    const unsigned q = elem_lanes(lane, __ballot_sync(FULL, e & 1), __ballot_sync(FULL, e & 2),
                                  __ballot_sync(FULL, e & 4));
    cr += __popc(q & mr);
    ca += __popc(q & ma);
    if (sorted) {
      const int pr = nr + __popc(mr & lt), pa = na + __popc(ma & lt);
      if (vr && pr < RAD_CAP) put(pr, va && pa < ANG_CAP ? pa : -1, j, dx, dy, dz, r, e);
      nr += __popc(mr);
      na += __popc(ma);
    }
  }
  if (lane >= NE) cr = ca = 0;
  int ir = cr, ia = ca;   // inclusive scan over lanes 0 .. NE; lane NE ends with the totals
#pragma unroll
  for (int o = 1; o < 8; o <<= 1) {
    const int vr = __shfl_up_sync(FULL, ir, o), va = __shfl_up_sync(FULL, ia, o);
    if (lane >= o) {
      ir += vr;
      ia += va;
    }
  }
  orr = ir - cr;
  oa = ia - ca;
  if (__shfl_sync(FULL, orr, NE) > RAD_CAP || __shfl_sync(FULL, oa, NE) > ANG_CAP) {
    if (lane == 0) post_status(st, FNN_E_CAPACITY, -(long long)(i + 1));
    return false;
  }
  if (!sorted) {   // pass 2: scatter into element segments (stable within an element)
    int runr = orr, runa = oa;    // lane q: next free radial / angular slot of element q
    for (int kb = k0; kb < k1; kb += 32) {
      int j, e;
      float dx, dy, dz, r;
      bool vr, va;
      entry(kb + lane, j, dx, dy, dz, r, e, vr, va);
      const unsigned mr = __ballot_sync(FULL, vr), ma = __ballot_sync(FULL, va);
      const unsigned b0 = __ballot_sync(FULL, e & 1), b1 = __ballot_sync(FULL, e & 2),
                     b2 = __ballot_sync(FULL, e & 4);
      const unsigned same = elem_lanes(e, b0, b1, b2), q = elem_lanes(lane, b0, b1, b2);
      const int br = __shfl_sync(FULL, runr, e), ba = __shfl_sync(FULL, runa, e);
      if (vr) put(br + __popc(same & mr & lt), va ? ba + __popc(same & ma & lt) : -1, j, dx, dy, dz, r, e);
      runr += __popc(q & mr);
      runa += __popc(q & ma);
    }
  }
  __syncwarp();
  return true;
}

// Stage atom i's neighbours for the forward (FwdNbr); returns false when the atom has no structure, or
// (after posting FNN_E_CAPACITY) when a list overflows.  The per-element counts are kept one element per
// lane: on return lane q < NE holds the start of element q's radial (orr) and angular (oa) segment and its
// angular count (ca); lane NE holds the totals in orr and oa.  A row sorted by neighbour element is staged
// in one pass, any other in two (count, then scatter, stable within an element).
__device__ bool stage_fwd(const StageArgs &A, const AevParams &P, int i, FwdNbr &S, int &orr, int &oa, int &ca,
                          DevStatus *st) {
  const int lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1u;
  const int mol = A.atom_mol[i];
  if (mol < 0) return false;   // atom outside every structure (already posted)
  const float4 pi = A.pos[i];
  const MolGrid &g = A.grid[mol];
  const int pbc = g.pbc;
  const float Lx = pbc ? g.Lx : 0.f, Ly = pbc ? g.Ly : 0.f, Lz = pbc ? g.Lz : 0.f;
  const int k0 = (int)min((int64_t)A.row_ptr[i], A.cap), k1 = (int)min((int64_t)A.row_ptr[i + 1], A.cap);
  struct Ent {
    float dx, dy, dz, r;
    int e;
    bool vr, va;
  };
  auto entry = [&](int k, Ent &t) {
    t.vr = t.va = false;
    t.e = 0;
    t.dx = t.dy = t.dz = t.r = 0.f;
    if (k < k1) {
      const int j = A.nbr[k];
      const char4 sh = A.shift[k];
      const float4 pj = A.pos[j];
      t.dx = (pj.x - pi.x) + (float)sh.x * Lx;
      t.dy = (pj.y - pi.y) + (float)sh.y * Ly;
      t.dz = (pj.z - pi.z) + (float)sh.z * Lz;
      t.r = sqrt_fast(t.dx * t.dx + t.dy * t.dy + t.dz * t.dz);
      t.vr = t.r < P.rc_rad;
      t.va = t.r < P.rc_ang;
      t.e = A.elem[j];
    }
  };
  auto put = [&](int pr, int pa, const Ent &t) {
    S.rr[pr] = make_float2(t.r, log2_fast(switch_f(P, t.r, P.rc_rad, P.inv_rc_rad)) - 2.f);
    if (pa >= 0) {
      const float ir = rcp_fast(t.r);
      S.au[pa] = make_float4(t.dx * ir, t.dy * ir, t.dz * ir, 0.5f * t.r);
      S.la[pa] = log2_fast(switch_f(P, t.r, P.rc_ang, P.inv_rc_ang)) + 0.5f;
    }
  };
  const bool mine = lane < NE;   // lane q counts element q
  int cr = 0;
  ca = 0;
  if (k1 - k0 <= A.sorted_upto) {   // one pass: the subsets of a sorted row are sorted
    int nr = 0, na = 0;
    for (int kb = k0; kb < k1; kb += 32) {
      Ent t;
      entry(kb + lane, t);
      const unsigned mr = __ballot_sync(FULL, t.vr), ma = __ballot_sync(FULL, t.va);
      const unsigned q = elem_lanes(lane, __ballot_sync(FULL, t.e & 1), __ballot_sync(FULL, t.e & 2),
                                    __ballot_sync(FULL, t.e & 4));
      cr += __popc(q & mr);
      ca += __popc(q & ma);
      const int pr = nr + __popc(mr & lt), pa = na + __popc(ma & lt);
      if (t.vr && pr < RAD_CAP) put(pr, t.va && pa < ANG_CAP ? pa : -1, t);
      nr += __popc(mr);
      na += __popc(ma);
    }
  } else {   // pass 1: counts per element
    for (int kb = k0; kb < k1; kb += 32) {
      Ent t;
      entry(kb + lane, t);
      const unsigned mr = __ballot_sync(FULL, t.vr), ma = __ballot_sync(FULL, t.va);
      const unsigned q = elem_lanes(lane, __ballot_sync(FULL, t.e & 1), __ballot_sync(FULL, t.e & 2),
                                    __ballot_sync(FULL, t.e & 4));
      cr += __popc(q & mr);
      ca += __popc(q & ma);
    }
  }
  if (!mine) cr = ca = 0;
  // exclusive scan over lanes 0 .. NE of the counts; lane NE receives the totals
  int ir = cr, ia = ca;
#pragma unroll
  for (int o = 1; o < 8; o <<= 1) {
    const int vr = __shfl_up_sync(FULL, ir, o), va = __shfl_up_sync(FULL, ia, o);
    if (lane >= o) {
      ir += vr;
      ia += va;
    }
  }
  orr = ir - cr;
  oa = ia - ca;
  if (__shfl_sync(FULL, orr, NE) > RAD_CAP || __shfl_sync(FULL, oa, NE) > ANG_CAP) {
    if (lane == 0) post_status(st, FNN_E_CAPACITY, -(long long)(i + 1));
    return false;
  }
  if (k1 - k0 > A.sorted_upto) {   // pass 2: scatter into element segments (stable within an element)
    int runr = orr, runa = oa;    // lane q: next free radial / angular slot of element q
    for (int kb = k0; kb < k1; kb += 32) {
      Ent t;
      entry(kb + lane, t);
      const unsigned mr = __ballot_sync(FULL, t.vr), ma = __ballot_sync(FULL, t.va);
      const unsigned b0 = __ballot_sync(FULL, t.e & 1), b1 = __ballot_sync(FULL, t.e & 2),
                     b2 = __ballot_sync(FULL, t.e & 4);
      const unsigned same = elem_lanes(t.e, b0, b1, b2), q = elem_lanes(lane, b0, b1, b2);
      const int br = __shfl_sync(FULL, runr, t.e), ba = __shfl_sync(FULL, runa, t.e);
      if (t.vr) put(br + __popc(same & mr & lt), t.va ? ba + __popc(same & ma & lt) : -1, t);
      runr += __popc(q & mr);
      runa += __popc(q & ma);
    }
  }
  __syncwarp();
  return true;
}

// slot block of the element pair (a, b), a <= b, in row-major upper-triangle order
__device__ __forceinline__ int pair_of(int a, int b) { return a * NE - a * (a - 1) / 2 + (b - a); }

template <typename OutT>
__device__ __forceinline__ void store_out(OutT *p, float v, float inv);
template <>
__device__ __forceinline__ void store_out<float>(float *p, float v, float) { *p = v; }
template <>
__device__ __forceinline__ void store_out<__nv_bfloat16>(__nv_bfloat16 *p, float v, float) { *p = __float2bfloat16(v); }
template <>   // fp8 e4m3 of v * inv, saturating
__device__ __forceinline__ void store_out<__nv_fp8_e4m3>(__nv_fp8_e4m3 *p, float v, float inv) {
  p->__x = __nv_cvt_float_to_fp8(v * inv, __NV_SATFINITE, __NV_E4M3);
}

struct AevFwdArgs {
  StageArgs sa;
  AevParams P;
  float *out;             // [rows][1008]
  __nv_bfloat16 *out_lo;  // low bf16 half of a split output, or NULL
  float out_inv;          // fp8 outputs hold aev * out_inv
  const int32_t *inv;     // padded row -> atom (-1 padding); NULL = rows are atoms
  const int32_t *meta;    // META_NPAD when inv != NULL
  int n_atoms;
  DevStatus *st;
};

// rounding residual of a bf16 store (the lo term of a hi / lo split)
__device__ __forceinline__ void store_lo(__nv_bfloat16 *lo, size_t c, float v) {
  if (lo) lo[c] = __float2bfloat16(v - __bfloat162float(__float2bfloat16(v)));
}

// zeros over n elements of type T from p (16-byte aligned; n * sizeof(T) a multiple of 16), by the warp
template <typename T>
__device__ __forceinline__ void zero_span(T *p, int n) {
  const int lane = threadIdx.x & 31;
  uint4 *q = reinterpret_cast<uint4 *>(p);
  const int n16 = n * (int)sizeof(T) / 16;
  for (int c = lane; c < n16; c += 32) q[c] = make_uint4(0u, 0u, 0u, 0u);
}

// The table of an atom's non-empty blocks from its per-element angular counts and starts (lane q < NE:
// ca, oa); lane p < NPAIR evaluates block p = (a, b).  Returns the slots (a multiple of four per block) and
// the number of blocks in nblk.
__device__ __forceinline__ int build_blocks(BlockTable &W, int ca, int oa, int &nblk) {
  const int lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1u;
  const int a = (lane >= 7) + (lane >= 13) + (lane >= 18) + (lane >= 22) + (lane >= 25) + (lane >= 27);
  const int b = min(a + lane - pair_of(a, a), NE - 1);
  const int na = __shfl_sync(FULL, ca, a), nb = __shfl_sync(FULL, ca, b);
  const int ja0 = __shfl_sync(FULL, oa, a), kb0 = __shfl_sync(FULL, oa, b);
  const int cnt = lane < NPAIR ? (a == b ? na * (na - 1) / 2 : na * nb) : 0;
  const unsigned nonempty = __ballot_sync(FULL, cnt > 0);
  int incl = (cnt + 3) & ~3;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int v = __shfl_up_sync(FULL, incl, o);
    if (lane >= o) incl += v;
  }
  const int T = __shfl_sync(FULL, incl, 31);
  if (cnt > 0) {
    const int e = __popc(nonempty & lt);
    W.bt[e] = make_int4(incl - ((cnt + 3) & ~3), ja0 | (kb0 << 8) | ((a == b) << 16), nb, na);
    W.bi[e] = rcp_fast((float)(a == b ? na : nb));
    W.bq[e] = lane | (cnt << 8);
  }
  nblk = __popc(nonempty);
  if (lane == 0) {
    W.bt[nblk] = make_int4(T, 0, 0, 0);
    W.bq[nblk] = 0;
    W.bi[nblk] = 0.f;
  }
  __syncwarp();
  return T;
}

// The pair of slot w of table entry idx (ja, ka: angular entries); false for a padding slot (ja = ka = 0)
__device__ __forceinline__ bool block_pair(const BlockTable &W, int idx, int w, int &ja, int &ka) {
  const int4 bk = W.bt[idx];
  const int cnt = W.bq[idx] >> 8;
  const bool diag = (bk.y >> 16) != 0;
  const int n = bk.w, dv = diag ? n : bk.z, D = (n - 1) >> 1;
  int q = (int)((float)w * W.bi[idx]);   // w / dv, corrected below
  if (q * dv > w) q--;
  else if ((q + 1) * dv <= w) q++;
  const int r = w - q * dv;
  const int j0 = bk.y & 0xff;
  int jrel, krel;
  if (diag) {
    const bool tail = q >= D;   // even n: the last diagonal, d = n / 2
    jrel = tail ? w - D * n : r;
    const int k = jrel + (tail ? n >> 1 : q + 1);
    krel = k < n ? k : k - n;
  } else {
    jrel = q;
    krel = ((bk.y >> 8) & 0xff) - j0 + r;
  }
  const bool real = w < cnt;
  ja = real ? j0 + jrel : 0;
  ka = real ? j0 + krel : 0;
  return real;
}

// Slot base + lane of one batch (32 consecutive slots in block order; every block padded to a multiple of
// four slots) for the lane: the table entry of its block (idx), its angular entries ja, ka, and whether it
// opens its block; false for a padding slot (ja = ka = 0 then).  cur is the table entry holding the
// batch's first slot (warp-uniform) and is advanced to the one holding its last; nblk the table's entries
// before the one-past-the-last.  Within a block of one element (n entries) the pairs run along cyclic
// diagonals {j, (j + d) mod n}, d = 1 .. n/2 (for even n the last diagonal holds n/2 pairs); within a block
// of two elements, j-major.
__device__ __forceinline__ bool batch_triplet(const BlockTable &W, int base, int nblk, int &cur, int &idx, int &ja,
                                              int &ka, bool &opens) {
  const int lane = threadIdx.x & 31;
  if (W.bt[cur + 1].x == base) cur++;   // a block opening at the batch's first slot
  // the blocks opening inside the batch, as bits of the slot offsets (table entries one per lane)
  unsigned bit = 0u;
  if (lane <= nblk) {
    const int o = W.bt[lane].x - base;
    if (o > 0 && o < 32) bit = 1u << o;
  }
  const unsigned M = __reduce_or_sync(FULL, bit);
  idx = cur + __popc(M & ((2u << lane) - 1u));
  cur += __popc(M);
  const int w = base + lane - W.bt[idx].x;
  opens = w == 0 && (W.bq[idx] >> 8) > 0;
  return block_pair(W, idx, w, ja, ka);
}

// The lane's triplet (angular entries ja, ka) into the batch rows: 4 section powers and 8 Gaussians; a
// padding slot's Gaussians are zero (its switch product -inf in the exponent)
__device__ __forceinline__ void produce_triplet(FwdStage &W, const AevParams &P, bool real, int ja, int ka) {
  const int lane = threadIdx.x & 31;
  const float4 u1 = W.nb.au[ja], u2 = W.nb.au[ka];
  const float c95 = 0.95f * (u1.x * u2.x + u1.y * u2.y + u1.z * u2.z);
  const float s95 = sqrt_fast(fmaxf(1.f - c95 * c95, 0.f));
  // sections (s, s + 1) and shifts (m, m + 1) side by side in packed pairs
  const float2 c2 = dup2(c95), s2 = dup2(s95), z2 = dup2(P.zeta);
#pragma unroll
  for (int s = 0; s < NSZ; s += 2) {
    const float2 base = fma2(s2, P.hsin2[s >> 1], fma2(c2, P.hcos2[s >> 1], dup2(0.5f)));
    const float2 f = exp2_2(mul2(z2, log2_2(base)));
    W.sf[s][lane] = f.x;
    W.sf[s + 1][lane] = f.y;
  }
  // the switch product 2 fc_j fc_k enters the exponent: 2^(-eta log2(e) dr^2 + log2(2 fc_j fc_k))
  const float rbar = u1.w + u2.w, lf = real ? W.nb.la[ja] + W.nb.la[ka] : __int_as_float(0xff800000);
  const float2 rb2 = dup2(rbar), lf2 = dup2(lf), ea2 = dup2(P.eta_a_l2);
#pragma unroll
  for (int m = 0; m < NSA; m += 2) {
    const float2 dr = add2(rb2, P.nsha2[m >> 1]);
    const float2 g = exp2_2(fma2(mul2(dr, dr), ea2, lf2));
    W.sg[m][lane] = g.x;
    W.sg[m + 1][lane] = g.y;
  }
}

// Where a row of the forward goes: a row of the AEV array in global memory (and of its low half when the
// output is split into bf16 hi + lo)
template <typename OutT>
struct GlobalRow {
  OutT *out;
  __nv_bfloat16 *lo;
  float inv;
  __device__ __forceinline__ void zero() const {
    zero_span(out, NAEV);
    if (lo) zero_span(lo, NAEV);
  }
  __device__ __forceinline__ void put(int c, float v) const {
    store_out<OutT>(out + c, v, inv);
    store_lo(lo, c, v);
  }
};

// Radial slots of a staged row: lane (h, k) sums the shift pair (2k, 2k + 1), packed, over every fourth
// neighbour (h) of each element segment; elements without neighbours are skipped (their slots hold zeros
// already) unless zeros is set
template <typename Sink>
__device__ __forceinline__ void radial_row(const AevParams &P, const FwdStage &W, const Sink &o, int orr, bool zeros) {
  const int lane = threadIdx.x & 31;
  const int h = lane >> 3, k = lane & 7;
  const float2 nR = P.nshr2[k], ce2 = dup2(P.eta_r_l2);
#pragma unroll 1
  for (int q = 0; q < NE; q++) {
    const int t0 = __shfl_sync(FULL, orr, q), t1 = __shfl_sync(FULL, orr, q + 1);
    if (t0 == t1 && !zeros) continue;
    int t = t0 + h;
    float2 a0 = make_float2(0.f, 0.f), a1 = a0;
    for (; t + 4 < t1; t += 8) {
      const float2 v0 = W.nb.rr[t], v1 = W.nb.rr[t + 4];
      const float2 d0 = add2(dup2(v0.x), nR), d1 = add2(dup2(v1.x), nR);
      a0 = add2(a0, exp2_2(fma2(mul2(d0, d0), ce2, dup2(v0.y))));
      a1 = add2(a1, exp2_2(fma2(mul2(d1, d1), ce2, dup2(v1.y))));
    }
    if (t < t1) {
      const float2 v0 = W.nb.rr[t];
      const float2 d0 = add2(dup2(v0.x), nR);
      a0 = add2(a0, exp2_2(fma2(mul2(d0, d0), ce2, dup2(v0.y))));
    }
    float2 acc = add2(a0, a1);
    acc = add2(acc, make_float2(__shfl_xor_sync(FULL, acc.x, 8), __shfl_xor_sync(FULL, acc.y, 8)));
    acc = add2(acc, make_float2(__shfl_xor_sync(FULL, acc.x, 16), __shfl_xor_sync(FULL, acc.y, 16)));
    if (h < 2) o.put(q * NSR + 2 * k + h, h ? acc.y : acc.x);
  }
}

// The AEV row of atom i (i < 0: a padding row of zeros) into o, by one warp staged in W
template <typename Sink>
__device__ __forceinline__ void aev_row(const AevFwdArgs &A, FwdStage &W, int i, const Sink &o) {
  const int lane = threadIdx.x & 31;
  const AevParams &P = A.P;
  int orr, oa, ca;
  const bool ok = i >= 0 && stage_fwd(A.sa, P, i, W.nb, orr, oa, ca, A.st);
  // every slot of an element (pair) without neighbours stays zero
  o.zero();
  __syncwarp();   // orders the zeros before the lanes' own stores below
  if (!ok) return;
  radial_row(P, W, o, orr, false);
  // ---- angular: every unordered pair j < k of the element-sorted angular list, 32 per batch,
  // enumerated block by block in slot order (element pair (a, b), a <= b), so a pair's 32 slots are
  // complete when its block ends.  The producer lane evaluates one triplet; lane (m, s) then sums
  // pow_s * gauss_m over the batch in four chains, which go to the output row when the block ends.
  {
    int nblk;
    const int T = build_blocks(W.tb, ca, oa, nblk);
    const int s_my = lane & 3, m_my = lane >> 2;
    const float *fr = W.sf[s_my], *gr = W.sg[m_my];
    int run_p = -1;          // slot block being summed (warp-uniform)
    float2 ra = make_float2(0.f, 0.f), rb = make_float2(0.f, 0.f);   // four chains as two packed pairs
    auto put = [&](int pp, float v) { o.put(NRAD + pp * 32 + lane, v); };
    auto open = [&](int pn) {
      if (run_p >= 0) put(run_p, (ra.x + ra.y) + (rb.x + rb.y));
      ra = rb = make_float2(0.f, 0.f);
      run_p = pn;
    };
    int cur = 0;
    for (int base = 0; base < T; base += 32) {
      // every lane evaluates a triplet; a padding slot's Gaussians are zero (its switch product -inf)
      int idx, ja, ka;
      bool opens;
      const bool real = batch_triplet(W.tb, base, nblk, cur, idx, ja, ka, opens);
      produce_triplet(W, P, real, ja, ka);
      if (opens) W.sp[lane] = W.tb.bq[idx] & 0xff;
      // blocks open only at slots that are multiples of four
      const unsigned starts = __ballot_sync(FULL, opens);
      __syncwarp();
#pragma unroll
      for (int q = 0; q < 32; q += 4) {
        const float4 fv = *reinterpret_cast<const float4 *>(fr + q);
        const float4 gv = *reinterpret_cast<const float4 *>(gr + q);
        if ((starts >> q) & 1u) open(W.sp[q]);
        ra = fma2(make_float2(fv.x, fv.y), make_float2(gv.x, gv.y), ra);
        rb = fma2(make_float2(fv.z, fv.w), make_float2(gv.z, gv.w), rb);
      }
      __syncwarp();
    }
    if (run_p >= 0) put(run_p, (ra.x + ra.y) + (rb.x + rb.y));
  }
}

// One warp's share of the forward: rows wg, wg + nw, ..., staged in W (the kernel below, and the fused
// small-system kernel, call it)
// (rl: when set, only the nrl rows rl[0 ..) -- atoms, without inv -- in place of every row)
template <typename OutT>
__device__ __forceinline__ void aev_forward_rows(const AevFwdArgs &A, FwdStage &W, int wg, int nw,
                                                 const int *rl = nullptr, int nrl = 0) {
  const int nrows = rl ? nrl : (A.inv ? A.meta[META_NPAD] : A.n_atoms);
  for (int q = wg; q < nrows; q += nw) {
    const int row = rl ? rl[q] : q;
    const GlobalRow<OutT> o{reinterpret_cast<OutT *>(A.out) + (size_t)row * NAEV,
                            A.out_lo ? A.out_lo + (size_t)row * NAEV : nullptr, A.out_inv};
    aev_row(A, W, A.inv && !rl ? A.inv[row] : row, o);
    __syncwarp();
  }
}

// The same rows with K warps per row (K > 1; for systems with fewer rows than warps): warp part 0 of a
// row writes the radial slots and the zeros of element pairs without triplets, parts 1 .. K-1 take the
// row's non-empty element-pair blocks in turn, each block's slots summed by one warp from its own batches
template <typename OutT>
__device__ void aev_forward_parts(const AevFwdArgs &A, FwdStage &W, int wg, int nw, int K, const int *rl = nullptr,
                                  int nrl = 0) {
  const int lane = threadIdx.x & 31;
  const AevParams &P = A.P;
  const int part = wg % K, groups = nw / K;
  if (wg >= groups * K) return;
  const int nrows = rl ? nrl : (A.inv ? A.meta[META_NPAD] : A.n_atoms);
  const int s_my = lane & 3, m_my = lane >> 2;
  const float *fr = W.sf[s_my], *gr = W.sg[m_my];
  for (int q = wg / K; q < nrows; q += groups) {
    const int row = rl ? rl[q] : q;
    OutT *out = reinterpret_cast<OutT *>(A.out) + (size_t)row * NAEV;
    __nv_bfloat16 *lo = A.out_lo ? A.out_lo + (size_t)row * NAEV : nullptr;
    const int i = A.inv && !rl ? A.inv[row] : row;
    int orr, oa, ca;
    const bool ok = i >= 0 && stage_fwd(A.sa, P, i, W.nb, orr, oa, ca, A.st);
    if (!ok) {
      if (part == 0) {
        for (int c = lane; c < NAEV; c += 32) {
          store_out<OutT>(out + c, 0.f, A.out_inv);
          store_lo(lo, c, 0.f);
        }
      }
      __syncwarp();
      continue;
    }
    int nblk;
    build_blocks(W.tb, ca, oa, nblk);
    if (part == 0) {
      radial_row(P, W, GlobalRow<OutT>{out, lo, A.out_inv}, orr, true);
      const unsigned present = __reduce_or_sync(FULL, lane < nblk ? 1u << (W.tb.bq[lane] & 0xff) : 0u);
      for (int pp = 0; pp < NPAIR; pp++)
        if (!((present >> pp) & 1u)) {
          store_out<OutT>(out + NRAD + pp * 32 + lane, 0.f, A.out_inv);
          store_lo(lo, NRAD + pp * 32 + lane, 0.f);
        }
    } else {
      for (int e = part - 1; e < nblk; e += K - 1) {
        const int s0 = W.tb.bt[e].x, s1 = W.tb.bt[e + 1].x, pb = W.tb.bq[e] & 0xff;
        float2 ra = make_float2(0.f, 0.f), rb = make_float2(0.f, 0.f);
        for (int base = s0; base < s1; base += 32) {
          int ja, ka;
          const bool real = block_pair(W.tb, e, base - s0 + lane, ja, ka);
          produce_triplet(W, P, real, ja, ka);
          __syncwarp();
#pragma unroll
          for (int q = 0; q < 32; q += 4) {
            const float4 fv = *reinterpret_cast<const float4 *>(fr + q);
            const float4 gv = *reinterpret_cast<const float4 *>(gr + q);
            ra = fma2(make_float2(fv.x, fv.y), make_float2(gv.x, gv.y), ra);
            rb = fma2(make_float2(fv.z, fv.w), make_float2(gv.z, gv.w), rb);
          }
          __syncwarp();
        }
        const float v = (ra.x + ra.y) + (rb.x + rb.y);
        store_out<OutT>(out + NRAD + pb * 32 + lane, v, A.out_inv);
        store_lo(lo, NRAD + pb * 32 + lane, v);
      }
    }
    __syncwarp();
  }
}

// Warps per row (1 to 8) for nrows rows on nw warps: the kernels are launched as one wave of resident blocks
// (up to eight warps' worth per row), and rows fewer than half the warps are each shared by several warps,
// since a row's work is serial within its warp (the 648 atoms of a water box on 4,736 warps would leave most
// of the GPU idle)
__device__ __forceinline__ int row_parts(int nrows, int nw) {
  const int k = nrows > 0 ? nw / nrows : 1;
  return k < 2 ? 1 : (k > 8 ? 8 : k);
}

template <typename OutT>
__global__ void __launch_bounds__(AEV_WARPS * 32, AEV_FWD_BLOCKS) k_aev_forward(AevFwdArgs A) {
  __shared__ FwdStage smem[AEV_WARPS];
  const int wl = threadIdx.x >> 5, nw = gridDim.x * AEV_WARPS;
  const int K = row_parts(A.inv ? A.meta[META_NPAD] : A.n_atoms, nw);
  if (K > 1)
    aev_forward_parts<OutT>(A, smem[wl], blockIdx.x * AEV_WARPS + wl, nw, K);
  else
    aev_forward_rows<OutT>(A, smem[wl], blockIdx.x * AEV_WARPS + wl, nw);
}

// ------------------------------------------------------------------- fused AEV -> first layer (BF16)
// The BF16 form's AEV and first layer in one kernel (section II.E: the networks read the AEV of each
// atomic centre): a persistent CTA per SM takes 64-row tiles of the species-sorted rows.  Its worker warps
// build the tile's AEV rows (the forward above, row by row) as bf16 straight into shared memory, in the
// tensor core's K-major 128-byte-swizzled layout; one thread then issues the tile's products with every
// member's first-layer weights (tcgen05.mma, M = 64, N = 256, weights streamed by TMA through a three-stage
// ring), and 16 of the workers apply bias + CELU to each member's accumulator as it completes and store h1.  The
// AEV never reaches global memory.  A 128-row tile would take 256 KB of shared memory as bf16, more than a
// CTA has, so the tiles are 64 rows: an M = 64 accumulator holds row r in TMEM lane 32 (r / 16) + r % 16.
// The AEV staging of the workers shares its space with the weight ring (the two phases of a tile do not
// overlap: a tile's AEV must be complete before its first product).
constexpr int FUSE_ROWS = 64;                 // rows of a tile (UMMA M)
constexpr int FUSE_WORKERS = 18;              // AEV warps; the first 16 are then the epilogue warps
constexpr int FUSE_EPI = 16;                  // (four per TMEM lane quarter)
constexpr int FUSE_THREADS = 32 * FUSE_WORKERS + 64;   // + the TMA warp and the MMA warp
constexpr int FUSE_KCH = 16;                  // 64-element K chunks of a row: 1008 columns padded to 1024
constexpr int FUSE_CHUNK = FUSE_ROWS * 128;   // bytes of one K chunk of the tile (8-row groups 1024 B apart)
constexpr int FUSE_BST = H1 * 128;            // one weight stage: 256 rows x 64 K elements
constexpr int FUSE_STAGES = 3;

struct FuseSmem {
  uint8_t A[FUSE_KCH * FUSE_CHUNK];           // the AEV tile, K chunk by K chunk (1024-byte aligned)
  union {
    uint8_t B[FUSE_STAGES][FUSE_BST];         // weight ring (products)
    FwdStage W[FUSE_WORKERS];                 // AEV staging (rows)
  } u;
  uint64_t full[FUSE_STAGES], empty[FUSE_STAGES], acc_full[2], acc_empty[2], fin;
  uint32_t tmem_base;
  int abort_flag;
  int next_row;                               // rows of the tile claimed by the workers
};
constexpr size_t fuse_smem_bytes() { return sizeof(FuseSmem) + 1024; }
static_assert(sizeof(FuseSmem) + 1024 <= (size_t)tc::SMEM_LIMIT, "fused kernel shared memory");

// Row r of the tile: column c at K chunk c / 64, byte 2 (c % 64) of the row's 128 bytes, 16-byte units
// XOR-swizzled by r % 8 (the pattern TMA's 128-byte swizzle writes and the descriptor reads)
struct TileRow {
  uint8_t *tile;
  int r;
  __device__ __forceinline__ void zero() const {
    const int lane = threadIdx.x & 31;
    for (int u = lane; u < FUSE_KCH * 8; u += 32)
      *reinterpret_cast<uint4 *>(tile + (u >> 3) * FUSE_CHUNK + r * 128 + (u & 7) * 16) = make_uint4(0u, 0u, 0u, 0u);
  }
  __device__ __forceinline__ void put(int c, float v) const {
    const int off = (c >> 6) * FUSE_CHUNK + r * 128 + ((((c >> 3) & 7) ^ (r & 7)) << 4) + ((c & 7) << 1);
    *reinterpret_cast<__nv_bfloat16 *>(tile + off) = __float2bfloat16(v);
  }
};

struct FuseArgs {
  AevFwdArgs aev;            // inv and meta give the padded species-sorted rows
  const int32_t *tile_elem;  // element of each 128-row tile (-1: none)
  long long rows_cap;        // rows of h1 (a multiple of 128)
  const float *bias;         // b1 [7][M * 256]
  __nv_bfloat16 *h1;         // [rows][M][256]
  int M;
};

__global__ void __launch_bounds__(FUSE_THREADS, 1) k_aev_l1(const __grid_constant__ CUtensorMap tmW1, FuseArgs p) {
  using namespace tc;
  extern __shared__ uint8_t smem_raw[];
  FuseSmem &S = *reinterpret_cast<FuseSmem *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  constexpr int WT = FUSE_WORKERS, WM = FUSE_WORKERS + 1;   // TMA warp, MMA warp
  volatile int *abort_flag = &S.abort_flag;
  const int M = p.M;
  const long long npad = min((long long)p.aev.meta[META_NPAD], p.rows_cap);
  const int ntile = (int)(npad / FUSE_ROWS);
  if (warp == WT && lane == 0) {
    for (int s = 0; s < FUSE_STAGES; s++) {
      mbar_init(&S.full[s], 1);
      mbar_init(&S.empty[s], 1);
    }
    for (int a = 0; a < 2; a++) {
      mbar_init(&S.acc_full[a], 1);
      mbar_init(&S.acc_empty[a], FUSE_EPI);   // one arrival per epilogue warp
    }
    mbar_init(&S.fin, 1);
    S.abort_flag = 0;
    fence_barrier_init();
  }
  if (warp == WM) {
    tmem_alloc(&S.tmem_base, 2 * H1);
    tmem_relinquish();
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = S.tmem_base;
  long long g = 0;   // weight stages issued (TMA lane) / consumed (MMA lane)
  int cnt = 0;       // accumulators issued (MMA lane) / drained (workers)
  for (int t = (int)blockIdx.x; t < ntile; t += (int)gridDim.x) {
    const int e = p.tile_elem[t >> 1];
    if (e < 0) continue;   // the whole CTA skips
    // ---- the tile's AEV rows, claimed one at a time by the workers
    if (threadIdx.x == 0) S.next_row = 0;
    __syncthreads();
    if (warp < WT) {
      for (;;) {
        int rr = 0;
        if (lane == 0) rr = atomicAdd(&S.next_row, 1);
        rr = __shfl_sync(FULL, rr, 0);
        if (rr >= FUSE_ROWS) break;
        const long long row = (long long)t * FUSE_ROWS + rr;
        aev_row(p.aev, S.u.W[warp], p.aev.inv[row], TileRow{S.A, rr});
        __syncwarp();
      }
      fence_proxy_async();   // the tile and the staging, written by threads, next read or overwritten by the async proxy
    }
    __syncthreads();
    if (*abort_flag) break;
    // ---- the products: one accumulator per member
    if (warp == WT) {
      if (lane == 0) {
        const long long g0 = g;
        for (int m = 0; m < M && !*abort_flag; m++)
          for (int kb = 0; kb < FUSE_KCH; kb++, g++) {
            const int s = (int)(g % FUSE_STAGES);
            if (g >= FUSE_STAGES && !mbar_wait(&S.empty[s], (uint32_t)(((g / FUSE_STAGES) - 1) & 1))) {
              *abort_flag = 1;
              break;
            }
            mbar_expect_tx(&S.full[s], (uint32_t)FUSE_BST);
            tma_load_3d(S.u.B[s], &tmW1, &S.full[s], kb * 64, m * H1, e);
          }
        // after an abort, every load issued must land before the ring is reused or the CTA exits
        if (*abort_flag)
          for (long long q = max(g0, g - FUSE_STAGES); q < g; q++)
            mbar_wait(&S.full[q % FUSE_STAGES], (uint32_t)((q / FUSE_STAGES) & 1));
      }
    } else if (warp == WM) {
      if (lane == 0) {
        const uint32_t idesc = idesc_bf16(FUSE_ROWS, H1), a0 = smem_u32(S.A);
        for (int m = 0; m < M && !*abort_flag; m++) {
          const int a = cnt & 1;
          if (cnt >= 2 && !mbar_wait(&S.acc_empty[a], (uint32_t)(((cnt >> 1) - 1) & 1))) {
            *abort_flag = 1;
            break;
          }
          fence_after();
          const uint32_t d = tmem + (uint32_t)(a * H1);
          for (int kb = 0; kb < FUSE_KCH; kb++, g++) {
            const int s = (int)(g % FUSE_STAGES);
            if (!mbar_wait(&S.full[s], (uint32_t)((g / FUSE_STAGES) & 1))) {
              *abort_flag = 1;
              break;
            }
            fence_after();
            const uint32_t b0 = smem_u32(S.u.B[s]);
#pragma unroll
            for (int k = 0; k < 4; k++)
              mma_bf16(d, sdesc_sw128(a0 + kb * FUSE_CHUNK + 32 * k), sdesc_sw128(b0 + 32 * k), idesc,
                       (kb | k) != 0 ? 1u : 0u);
            mma_commit(&S.empty[s]);
          }
          if (*abort_flag) break;
          mma_commit(&S.acc_full[a]);
          cnt++;
        }
      }
    } else if (warp < FUSE_EPI) {   // bias + CELU of each member's accumulator, rows of lane quarter q, 64 columns each
      const int q = warp & 3, part = warp >> 2;
      const long long row = (long long)t * FUSE_ROWS + q * 16 + (lane & 15);
      for (int m = 0; m < M; m++) {
        const int a = cnt & 1;
        const bool ok = mbar_wait(&S.acc_full[a], (uint32_t)((cnt >> 1) & 1));
        fence_after();
        if (!__all_sync(FULL, ok)) {
          *abort_flag = 1;
          break;
        }
        const uint32_t tb = tmem + (uint32_t)(a * H1) + ((uint32_t)(q * 32) << 16);
        const float *bias = p.bias + (long long)e * M * H1 + m * H1;
        __nv_bfloat16 *out = p.h1 + (row * M + m) * H1;
#pragma unroll 1
        for (int c = part * 64; c < part * 64 + 64; c += 16) {
          float v[16];
          tmem_ld16(tb + c, v);   // lanes 16..31 of the quarter hold no rows of an M = 64 accumulator
          if (lane < 16) {
            alignas(16) __nv_bfloat16 hb[16];
#pragma unroll
            for (int j = 0; j < 16; j += 4) {
              const float4 bb = __ldg(reinterpret_cast<const float4 *>(bias + c + j));
              hb[j] = __float2bfloat16(celu_f(v[j] + bb.x));
              hb[j + 1] = __float2bfloat16(celu_f(v[j + 1] + bb.y));
              hb[j + 2] = __float2bfloat16(celu_f(v[j + 2] + bb.z));
              hb[j + 3] = __float2bfloat16(celu_f(v[j + 3] + bb.w));
            }
            reinterpret_cast<uint4 *>(out + c)[0] = reinterpret_cast<const uint4 *>(hb)[0];
            reinterpret_cast<uint4 *>(out + c)[1] = reinterpret_cast<const uint4 *>(hb)[1];
          }
        }
        // the accumulator may be overwritten once every worker has read it
        fence_before();
        __syncwarp();
        if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&S.acc_empty[a])) : "memory");
        cnt++;
      }
    }
    // every product of the tile has completed (the workers drained the last accumulator) before its AEV
    // tile and the ring are overwritten by the next tile's rows
    __syncthreads();
    if (*abort_flag) break;
  }
  // every issued product must be complete before the TMEM is released (after an abort, MMAs may remain)
  if (warp == WM && lane == 0) {
    mma_commit(&S.fin);
    if (!mbar_wait(&S.fin, 0)) *abort_flag = 1;
  }
  fence_before();
  __syncthreads();
  if (*abort_flag && threadIdx.x == 0) post_status(p.aev.st, FNN_E_TIMEOUT, blockIdx.x);
  if (warp == WM) {
    fence_after();
    tmem_dealloc(tmem, 2 * H1);
  }
}

// ------------------------------------------------------------------------------------- adjoint
struct AevAdjArgs {
  StageArgs sa;
  AevParams P;
  const float *gaev;      // [rows][1008] dE/dAEV
  const int32_t *inv;     // padded row -> atom; NULL = rows are atoms
  const int32_t *meta;
  int n_atoms;
  float *F;               // [N][3], accumulated (caller zeroes)
  double *virial;         // [n_mol][9] accumulated, or NULL
  DevStatus *st;
};

// The dE/dAEV row is read through the L1 cache where it is used (4 KB per atom, re-read by the warp's
// lanes): staging it in shared memory would cap the number of resident warps.
// One warp's share of the adjoint: rows wg, wg + nw, ..., staged in W
// With K > 1 warps per row (systems with fewer rows than warps) warp part 0 of a row takes its radial
// terms and parts 1 .. K-1 its angular batches in turn; each warp scatters what it summed (the forces and
// virials are sums).
__device__ __forceinline__ void aev_adjoint_rows(const AevAdjArgs &A, AdjStage &W, int wg, int nw, int K = 1,
                                                 const int *rl = nullptr, int nrl = 0) {
  int lane = threadIdx.x & 31;
  NbrStage &S = W.nb;
  const AevParams &P = A.P;
  const int nrows = rl ? nrl : (A.inv ? A.meta[META_NPAD] : A.n_atoms);
  double *vacc = W.vacc;
  if (lane == 0)
    for (int q = 0; q < 9; q++) vacc[q] = 0.0;
  int cur_mol = -1;
  const int part = wg % K, groups = nw / K;
  if (wg >= groups * K) return;
  const bool do_rad = part == 0, do_ang = K == 1 || part > 0;
  const int apart = K == 1 ? 0 : part - 1, aparts = K == 1 ? 1 : K - 1;   // this warp's share of the batches
  for (int q = wg / K; q < nrows; q += groups) {
    const int row = rl ? rl[q] : q;
    const int i = A.inv && !rl ? A.inv[row] : row;
    if (i < 0) continue;
    const float *G = A.gaev + (size_t)row * NAEV;
    int orr, oa, cr, ca;
    if (!stage_neighbors(A.sa, P, i, S, orr, oa, cr, ca, A.st)) continue;
    // the angular part of the dE/dAEV row into shared memory while the radial terms run
    if (do_ang) {
      for (int c = lane; c < NPAIR * 8; c += 32) cp16(W.gs + (c >> 3) * GS_STRIDE + 4 * (c & 7), G + NRAD + 4 * c);
      cp_commit();
    }
    __syncwarp();
    // ---- radial: lane per entry, dE/dr = sum_k G[e*16+k] dT_k/dr
    const int nrad = __shfl_sync(FULL, orr, NE);
    if (!do_rad)
      for (int t = lane; t < nrad; t += 32) W.gacc[t][0] = W.gacc[t][1] = W.gacc[t][2] = 0.f;
    for (int t = lane; do_rad && t < nrad; t += 32) {
      const float4 d = S.rd[t];
      const float r = d.w;
      const float4 *Ge = reinterpret_cast<const float4 *>(G + S.re[t] * NSR);
      // 1/4 (g_k)' fc + 1/4 g_k fc' with g_k = exp(-eta (r - R_k)^2): g_k (fc' / 4 - eta dr_k fc / 2)
      const float fc2 = -0.5f * P.eta_r * switch_f(P, r, P.rc_rad, P.inv_rc_rad);
      const float dfc4 = 0.25f * switch_df(P, r, P.rc_rad, P.inv_rc_rad, P.pi_rc_rad);
      // shifts k and k + 1 side by side in packed pairs
      const float2 r2 = dup2(r), fc22 = dup2(fc2), dfc42 = dup2(dfc4), ce2 = dup2(P.eta_r_l2);
      float2 acc = make_float2(0.f, 0.f);
      auto term = [&](float2 Gk, int k) {
        const float2 dr = add2(r2, P.nshr2[k >> 1]);
        acc = fma2(mul2(Gk, exp2_2(mul2(mul2(dr, dr), ce2))), fma2(dr, fc22, dfc42), acc);
      };
#pragma unroll
      for (int k4 = 0; k4 < NSR / 4; k4++) {
        const float4 gv = __ldg(Ge + k4);
        term(make_float2(gv.x, gv.y), 4 * k4);
        term(make_float2(gv.z, gv.w), 4 * k4 + 2);
      }
      const float dEdr = acc.x + acc.y;
      const float f = dEdr * rcp_fast(r);
      W.gacc[t][0] = f * d.x;
      W.gacc[t][1] = f * d.y;
      W.gacc[t][2] = f * d.z;
    }
    __syncwarp();
    // ---- angular: one triplet per lane, enumerated by cyclic diagonals: diagonal d (1 <= d <= (n-1)/2)
    // holds the n pairs {j, (j + d) mod n}, and for even n the last one (d = n/2) the n/2 pairs with
    // j < n/2, so every pair appears once and within one diagonal the lanes hold distinct j and distinct k.
    // Up to 32 entries, lane e owns entry e's dE/dd in registers: for each diagonal a batch spans, it takes
    // its contribution as j from the lane of pair {e, e + d} and as k from the lane of pair {e - d, e}.
    // Beyond 32 entries the contributions go to shared memory by atomics (a batch spans at most 32/n + 2
    // diagonals, so an entry's atomics collide at most that often).
    {
      const int n = __shfl_sync(FULL, oa, NE);
      const int T = n * (n - 1) / 2;
      const int D = (n - 1) >> 1;      // diagonals of n pairs
      const float inv_n = rcp_fast((float)n);
      // t / n for 0 <= t < 2016, n <= 64
      auto div_n = [&](int t) {
        int q = (int)((float)t * inv_n);
        if (q * n > t) q--;
        else if ((q + 1) * n <= t) q++;
        return q;
      };
      const bool own = n <= 32;
      float ax = 0.f, ay = 0.f, az = 0.f;   // lane e < n: entry e (own)
      if (do_ang) cp_wait0();
      __syncwarp();
      for (int base = 32 * apart; do_ang && base < T; base += 32 * aparts) {
        const int t = min(base + lane, T - 1);
        int d, jc;
        if (t < D * n) {
          d = div_n(t);
          jc = t - d * n;
          d++;
        } else {                        // even n: d = n / 2, j < n / 2
          d = n >> 1;
          jc = t - D * n;
        }
        const int kc = jc + d < n ? jc + d : jc + d - n;
        const int ja = min(jc, kc), ka = max(jc, kc);   // list order: e(ja) <= e(ka)
        const int p = pair_of(S.ae[ja], S.ae[ka]);
        const float *Gp = W.gs + p * GS_STRIDE;
        const int rj1 = S.aidx[ja], rj2 = S.aidx[ka];
        const float4 d1 = S.rd[rj1], d2 = S.rd[rj2];
        const float r1 = d1.w, r2 = d2.w;
        const float ir1 = rcp_fast(r1), ir2 = rcp_fast(r2), inv12 = ir1 * ir2;
        const float c = (d1.x * d2.x + d1.y * d2.y + d1.z * d2.z) * inv12;
        const float c95 = 0.95f * c;
        const float s95 = sqrt_fast(fmaxf(1.f - c95 * c95, 0.f));
        const float ds95 = -0.9025f * c * rcp_fast(s95);   // d s95 / dc; s95 >= sqrt(1 - 0.95^2)
        // sections s and s + 1 side by side in packed pairs
        float fs[NSZ], dfs[NSZ];
        {
          const float2 c2 = dup2(c95), s2 = dup2(s95), d2 = dup2(ds95), z2 = dup2(P.zeta);
#pragma unroll
          for (int s = 0; s < NSZ; s += 2) {
            const float2 base = fma2(s2, P.hsin2[s >> 1], fma2(c2, P.hcos2[s >> 1], dup2(0.5f)));
            const float2 f = exp2_2(mul2(z2, log2_2(base)));
            // d f / d c = zeta f / base * 0.5 (0.95 cos + ds95 sin)
            const float2 df = mul2(mul2(mul2(z2, f), rcp_2(base)), fma2(d2, P.hsin2[s >> 1], P.qcos2[s >> 1]));
            fs[s] = f.x;
            fs[s + 1] = f.y;
            dfs[s] = df.x;
            dfs[s + 1] = df.y;
          }
        }
        const float rbar = 0.5f * (r1 + r2);
        // H_s = sum_m G[m][s] g_m and Hd_s = sum_m G[m][s] dr_m g_m (times -2 eta below: d g_m / d rbar); the
        // Gaussians of shifts (m, m + 1) in packed pairs, the sums scalar (packed sums over shift pairs need the
        // row transposed in shared memory, which cost more than they saved)
        float H[NSZ] = {0, 0, 0, 0}, Hd[NSZ] = {0, 0, 0, 0};
        {
          const float2 rb2 = dup2(rbar), ea2 = dup2(P.eta_a_l2);
#pragma unroll
          for (int m = 0; m < NSA; m += 2) {
            const float2 dr = add2(rb2, P.nsha2[m >> 1]);
            const float2 gm = exp2_2(mul2(mul2(dr, dr), ea2));
            const float2 tm = mul2(dr, gm);
            const float4 ga = *reinterpret_cast<const float4 *>(Gp + m * NSZ);
            const float4 gb = *reinterpret_cast<const float4 *>(Gp + (m + 1) * NSZ);
            H[0] += ga.x * gm.x; H[1] += ga.y * gm.x; H[2] += ga.z * gm.x; H[3] += ga.w * gm.x;
            Hd[0] += ga.x * tm.x; Hd[1] += ga.y * tm.x; Hd[2] += ga.z * tm.x; Hd[3] += ga.w * tm.x;
            H[0] += gb.x * gm.y; H[1] += gb.y * gm.y; H[2] += gb.z * gm.y; H[3] += gb.w * gm.y;
            Hd[0] += gb.x * tm.y; Hd[1] += gb.y * tm.y; Hd[2] += gb.z * tm.y; Hd[3] += gb.w * tm.y;
          }
        }
        const float f1 = S.afc[ja], f2 = S.afc[ka], df1 = S.adfc[ja], df2 = S.adfc[ka];
        // a lane past the last pair contributes nothing (its switch product taken as zero)
        const float C = base + lane < T ? f1 * f2 : 0.f, Cs = base + lane < T ? 1.f : 0.f;
        float sH = 0.f, sdH = 0.f, sHd = 0.f;
#pragma unroll
        for (int s = 0; s < NSZ; s++) {
          sH += fs[s] * H[s];
          sdH += dfs[s] * H[s];
          sHd += fs[s] * Hd[s];
        }
        const float dEdc = 2.f * C * sdH;
        const float dEdrbar = -4.f * P.eta_a * C * sHd;
        const float dEdC = 2.f * Cs * sH;
        const float dEdr1 = 0.5f * dEdrbar + dEdC * df1 * f2;
        const float dEdr2 = 0.5f * dEdrbar + dEdC * f1 * df2;
        const float a1 = (dEdr1 - dEdc * c * ir1) * ir1, b1 = dEdc * inv12;
        const float a2 = (dEdr2 - dEdc * c * ir2) * ir2;
        // entry ja gets g1, entry ka gets g2: by the cyclic roles, entry jc gets cj and entry kc gets ck
        const float g1x = a1 * d1.x + b1 * d2.x, g1y = a1 * d1.y + b1 * d2.y, g1z = a1 * d1.z + b1 * d2.z;
        const float g2x = a2 * d2.x + b1 * d1.x, g2y = a2 * d2.y + b1 * d1.y, g2z = a2 * d2.z + b1 * d1.z;
        const bool jfirst = jc == ja;
        const float cjx = jfirst ? g1x : g2x, cjy = jfirst ? g1y : g2y, cjz = jfirst ? g1z : g2z;
        const float ckx = jfirst ? g2x : g1x, cky = jfirst ? g2y : g1y, ckz = jfirst ? g2z : g1z;
        if (own) {
          // the diagonals of this batch, segment by segment: lanes [la, lb) hold diagonal dd with j = s0 + (lane - la)
          const int tend = min(base + 32, T);
          for (int ts = base; ts < tend;) {   // warp-uniform
            int dd, s0, tnext;
            if (ts < D * n) {
              const int q = div_n(ts);
              dd = q + 1;
              s0 = ts - q * n;
              tnext = dd * n;
            } else {
              dd = n >> 1;
              s0 = ts - D * n;
              tnext = T;
            }
            const int la = ts - base, lb = min(tnext, tend) - base;
            // as j: pair {e, e + dd}; as k: pair {e - dd, e} (no wrap on the last diagonal of even n)
            int jk = lane - dd;
            if (ts < D * n && jk < 0) jk += n;
            const int lj = la + lane - s0, lk = la + jk - s0;
            const bool vj = lane < n && lane >= s0 && lj < lb, vk = lane < n && jk >= s0 && lk < lb;
            const int sj = vj ? lj : 0, sk = vk ? lk : 0;
            const float xj = __shfl_sync(FULL, cjx, sj), yj = __shfl_sync(FULL, cjy, sj), zj = __shfl_sync(FULL, cjz, sj);
            const float xk = __shfl_sync(FULL, ckx, sk), yk = __shfl_sync(FULL, cky, sk), zk = __shfl_sync(FULL, ckz, sk);
            if (vj) {
              ax += xj;
              ay += yj;
              az += zj;
            }
            if (vk) {
              ax += xk;
              ay += yk;
              az += zk;
            }
            ts = lb + base;
          }
        } else if (base + lane < T) {
          const int rjc = S.aidx[jc], rkc = S.aidx[kc];   // distinct angular entries, distinct radial entries
          atomicAdd(&W.gacc[rjc][0], cjx);
          atomicAdd(&W.gacc[rjc][1], cjy);
          atomicAdd(&W.gacc[rjc][2], cjz);
          atomicAdd(&W.gacc[rkc][0], ckx);
          atomicAdd(&W.gacc[rkc][1], cky);
          atomicAdd(&W.gacc[rkc][2], ckz);
        }
      }
      __syncwarp();
      if (own && lane < n) {   // distinct angular entries are distinct radial entries
        const int rj = S.aidx[lane];
        W.gacc[rj][0] += ax;
        W.gacc[rj][1] += ay;
        W.gacc[rj][2] += az;
      }
    }
    __syncwarp();
    // ---- scatter: F_j -= g, F_i += sum g, W -= d (x) g
    float ci[3] = {0, 0, 0};
    float w[9];
#pragma unroll
    for (int q = 0; q < 9; q++) w[q] = 0.f;
    for (int t = lane; t < nrad; t += 32) {
      float g0 = W.gacc[t][0], g1 = W.gacc[t][1], g2 = W.gacc[t][2];
      if (K > 1 && g0 == 0.f && g1 == 0.f && g2 == 0.f) continue;   // not this part's entry
      int j = S.rj[t];
      atomicAdd(&A.F[3 * (size_t)j + 0], -g0);
      atomicAdd(&A.F[3 * (size_t)j + 1], -g1);
      atomicAdd(&A.F[3 * (size_t)j + 2], -g2);
      ci[0] += g0; ci[1] += g1; ci[2] += g2;
      float4 d = S.rd[t];
      float dv[3] = {d.x, d.y, d.z}, gv[3] = {g0, g1, g2};
#pragma unroll
      for (int x = 0; x < 3; x++)
#pragma unroll
        for (int y = 0; y < 3; y++) w[3 * x + y] -= dv[x] * gv[y];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
      for (int x = 0; x < 3; x++) ci[x] += __shfl_xor_sync(FULL, ci[x], o);
#pragma unroll
      for (int q = 0; q < 9; q++) w[q] += __shfl_xor_sync(FULL, w[q], o);
    }
    if (lane == 0) {
      atomicAdd(&A.F[3 * (size_t)i + 0], ci[0]);
      atomicAdd(&A.F[3 * (size_t)i + 1], ci[1]);
      atomicAdd(&A.F[3 * (size_t)i + 2], ci[2]);
      if (A.virial) {
        int mol = A.sa.atom_mol[i];
        if (mol != cur_mol) {
          if (cur_mol >= 0)
            for (int q = 0; q < 9; q++) atomicAdd(&A.virial[9 * (size_t)cur_mol + q], vacc[q]);
          for (int q = 0; q < 9; q++) vacc[q] = 0.0;
          cur_mol = mol;
        }
        for (int q = 0; q < 9; q++) vacc[q] += (double)w[q];
      }
    }
    __syncwarp();
  }
  if (lane == 0 && A.virial && cur_mol >= 0)
    for (int q = 0; q < 9; q++) atomicAdd(&A.virial[9 * (size_t)cur_mol + q], vacc[q]);
}

__global__ void __launch_bounds__(ADJ_WARPS * 32, AEV_ADJ_BLOCKS) k_aev_adjoint(AevAdjArgs A) {
  __shared__ AdjStage smem[ADJ_WARPS];
  // (one warp per row: splitting rows as the forward does measured slower here, 20.6 -> 29 us on a 648-atom
  // box, each part staging the whole row and scattering its own forces)
  const int wl = threadIdx.x >> 5;
  aev_adjoint_rows(A, smem[wl], blockIdx.x * ADJ_WARPS + wl, gridDim.x * ADJ_WARPS);
}

// ------------------------------------------------------------------------------- tangent (JVP)
// t = (dAEV/dx) . V: the directional derivative of every AEV entry along a displacement field V.
// Radial: d/dt [T_k(r)] = T_k'(r) rdot, rdot = d.(v_j - v_i) / r.  Angular: with c = cos theta,
// cdot = (d2.vd1 + d1.vd2) / (r1 r2) - c (r1dot / r1 + r2dot / r2),
// d/dt [2 f_s g_m C] = fdot_s (2 g_m C) + f_s (2 (gdot_m C + g_m Cdot)).  The forward's block table and
// batches (blocks padded to four slots): the producer lane stages one triplet's f_s, fdot_s, 2 g_m C and
// 2 (gdot_m C + g_m Cdot); lane (m, s) sums the two products over the batch in chains that go to the
// output row when the pair's block ends.
struct TanStage {
  NbrStage nb;
  float4 rv[RAD_CAP];            // v_j - v_i, rdot
  union {
    float2 rt[RAD_CAP];          // fc(r) rdot, fc'(r) rdot   (radial switch: the radial terms only)
    struct {                     // one batch of triplets, triplet innermost
      alignas(16) float sf[NSZ][SROW];
      alignas(16) float sfd[NSZ][SROW];
      alignas(16) float sg[NSA][SROW];
      alignas(16) float sgd[NSA][SROW];
      int sp[32];                // slot block of a triplet that opens one
    } b;
  };
  BlockTable tb;
};

struct AevTanArgs {
  StageArgs sa;
  AevParams P;
  const float *V;         // [N][3] displacement field
  void *out;              // [rows][1008], float or bf16
  __nv_bfloat16 *out_fwd; // the AEV rows themselves (bf16), or NULL: k_aev_forward's sums in its order (its
                          // Gaussians there as exp(-eta dr^2) times the switch product)
  const int32_t *inv;     // padded row -> atom; NULL = rows are atoms
  const int32_t *meta;
  int n_atoms;
  DevStatus *st;
};

constexpr int TAN_WARPS = 4, TAN_BLOCKS = 5;   // 11 KB of staging per warp

template <typename OutT>
__global__ void __launch_bounds__(TAN_WARPS * 32, TAN_BLOCKS) k_aev_tangent(AevTanArgs A) {
  __shared__ TanStage smem[TAN_WARPS];
  int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
  TanStage &W = smem[wl];
  NbrStage &S = W.nb;
  const AevParams &P = A.P;
  int nrows = A.inv ? A.meta[META_NPAD] : A.n_atoms;
  int wg = blockIdx.x * TAN_WARPS + wl, nw = gridDim.x * TAN_WARPS;
  for (int row = wg; row < nrows; row += nw) {
    OutT *out = reinterpret_cast<OutT *>(A.out) + (size_t)row * NAEV;
    int i = A.inv ? A.inv[row] : row;
    int orr, oa, cr, ca;
    bool ok = i >= 0 && stage_neighbors(A.sa, P, i, S, orr, oa, cr, ca, A.st);
    int off_r[NE + 1];   // radial segment starts, warp-uniform
#pragma unroll
    for (int q = 0; q <= NE; q++) off_r[q] = __shfl_sync(FULL, orr, q);
    __nv_bfloat16 *fout = A.out_fwd ? A.out_fwd + (size_t)row * NAEV : nullptr;
    if (!ok) {
      for (int c = lane; c < NAEV; c += 32) {
        store_out<OutT>(out + c, 0.f, 1.f);
        if (fout) fout[c] = __float2bfloat16(0.f);
      }
      __syncwarp();
      continue;
    }
    const float vix = A.V[3 * (size_t)i], viy = A.V[3 * (size_t)i + 1], viz = A.V[3 * (size_t)i + 2];
    const int nrad = off_r[NE];
    for (int t = lane; t < nrad; t += 32) {
      const int j = S.rj[t];
      const float4 d = S.rd[t];
      const float vx = A.V[3 * (size_t)j] - vix, vy = A.V[3 * (size_t)j + 1] - viy, vz = A.V[3 * (size_t)j + 2] - viz;
      const float rdot = (d.x * vx + d.y * vy + d.z * vz) * rcp_fast(d.w);
      W.rv[t] = make_float4(vx, vy, vz, rdot);
      const float dfc = switch_df(P, d.w, P.rc_rad, P.inv_rc_rad, P.pi_rc_rad);
      W.rt[t] = make_float2(switch_f(P, d.w, P.rc_rad, P.inv_rc_rad) * rdot, dfc * rdot);
    }
    __syncwarp();
    // ---- radial
    {
      int h = lane >> 4, k = lane & 15;
      float Rk = P.shf_r[k];
#pragma unroll 1
      for (int q = 0; q < NE; q++) {
        float acc = 0.f, accf = 0.f;
        for (int t = off_r[q] + h; t < off_r[q + 1]; t += 2) {
          const float dr = S.rd[t].w - Rk;
          const float2 ft = W.rt[t];
          const float gk = exp2f_fast(dr * dr * P.eta_r_l2);
          acc += gk * (-2.f * P.eta_r * dr * ft.x + ft.y);
          accf += gk * switch_f(P, S.rd[t].w, P.rc_rad, P.inv_rc_rad);
        }
        acc += __shfl_xor_sync(FULL, acc, 16);
        accf += __shfl_xor_sync(FULL, accf, 16);
        if (lane < 16) {
          store_out<OutT>(out + q * NSR + k, 0.25f * acc, 1.f);
          if (fout) fout[q * NSR + k] = __float2bfloat16(0.25f * accf);
        }
      }
    }
    __syncwarp();   // the batch rows below reuse the radial staging
    // ---- angular (the slots of element pairs without triplets are written as zeros up front)
    for (int c = lane; c < NPAIR * 32; c += 32) {
      store_out<OutT>(out + NRAD + c, 0.f, 1.f);
      if (fout) fout[NRAD + c] = __float2bfloat16(0.f);
    }
    __syncwarp();
    {
      const int s_my = lane & 3, m_my = lane >> 2;
      int nblk;
      const int T = build_blocks(W.tb, ca, oa, nblk);
      int run_p = -1;
      // four chains each, as two packed pairs: the tangent sums of the running block and (fout) its forward sums
      float2 ra = make_float2(0.f, 0.f), rb = ra, qa = ra, qb = ra;
      auto open = [&](int pn) {
        if (run_p >= 0) {
          store_out<OutT>(out + NRAD + run_p * 32 + lane, (ra.x + ra.y) + (rb.x + rb.y), 1.f);
          if (fout) fout[NRAD + run_p * 32 + lane] = __float2bfloat16((qa.x + qa.y) + (qb.x + qb.y));
        }
        ra = rb = qa = qb = make_float2(0.f, 0.f);
        run_p = pn;
      };
      const float *fr = W.b.sf[s_my], *fdr = W.b.sfd[s_my], *gr = W.b.sg[m_my], *gdr = W.b.sgd[m_my];
      int cur = 0;
      for (int base = 0; base < T; base += 32) {
        // every lane evaluates a triplet; a padding slot's switch product and its rate are zero
        int idx, ja, ka;
        bool opens;
        const bool real = batch_triplet(W.tb, base, nblk, cur, idx, ja, ka, opens);
        {
          const int rj1 = S.aidx[ja], rj2 = S.aidx[ka];
          const float4 d1 = S.rd[rj1], d2 = S.rd[rj2], v1 = W.rv[rj1], v2 = W.rv[rj2];
          const float r1 = d1.w, r2 = d2.w, ir1 = rcp_fast(r1), ir2 = rcp_fast(r2), inv12 = ir1 * ir2;
          const float c = (d1.x * d2.x + d1.y * d2.y + d1.z * d2.z) * inv12;
          const float cdot = (d2.x * v1.x + d2.y * v1.y + d2.z * v1.z + d1.x * v2.x + d1.y * v2.y + d1.z * v2.z) * inv12 -
                             c * (v1.w * ir1 + v2.w * ir2);
          const float c95 = 0.95f * c;
          const float s95 = sqrt_fast(fmaxf(1.f - c95 * c95, 0.f));
          const float ds95 = -0.9025f * c * rcp_fast(s95);
          const float zc = P.zeta * cdot;
          // sections (s, s + 1) and shifts (m, m + 1) side by side in packed pairs
          const float2 c2p = dup2(c95), s2p = dup2(s95), d2p = dup2(ds95), z2 = dup2(P.zeta), zc2 = dup2(zc);
#pragma unroll
          for (int sidx = 0; sidx < NSZ; sidx += 2) {
            const float2 base = fma2(s2p, P.hsin2[sidx >> 1], fma2(c2p, P.hcos2[sidx >> 1], dup2(0.5f)));
            const float2 f = exp2_2(mul2(z2, log2_2(base)));
            // fdot = zeta f / base * 0.5 (0.95 cos + ds95 sin) * cdot
            const float2 fd = mul2(mul2(mul2(zc2, f), rcp_2(base)), fma2(d2p, P.hsin2[sidx >> 1], P.qcos2[sidx >> 1]));
            W.b.sf[sidx][lane] = f.x;
            W.b.sf[sidx + 1][lane] = f.y;
            W.b.sfd[sidx][lane] = fd.x;
            W.b.sfd[sidx + 1][lane] = fd.y;
          }
          const float rbar = 0.5f * (r1 + r2), rbdot = 0.5f * (v1.w + v2.w);
          const float f1 = S.afc[ja], f2 = S.afc[ka];
          const float C = real ? f1 * f2 : 0.f;
          const float Cdot = real ? S.adfc[ja] * v1.w * f2 + f1 * S.adfc[ka] * v2.w : 0.f;
          // 2 g C and 2 (gdot C + g Cdot) = g (dr (-4 eta rbdot C) + 2 Cdot), gdot = -2 eta dr g rbdot
          const float C2 = 2.f * C, a2 = -4.f * P.eta_a * rbdot * C, c2 = 2.f * Cdot;
          const float2 rb2 = dup2(rbar), ea2 = dup2(P.eta_a_l2), C22 = dup2(C2), a22 = dup2(a2), c22 = dup2(c2);
#pragma unroll
          for (int m = 0; m < NSA; m += 2) {
            const float2 dr = add2(rb2, P.nsha2[m >> 1]);
            const float2 g = exp2_2(mul2(mul2(dr, dr), ea2));
            const float2 gc = mul2(g, C22), gd = mul2(g, fma2(dr, a22, c22));
            W.b.sg[m][lane] = gc.x;
            W.b.sg[m + 1][lane] = gc.y;
            W.b.sgd[m][lane] = gd.x;
            W.b.sgd[m + 1][lane] = gd.y;
          }
          if (opens) W.b.sp[lane] = W.tb.bq[idx] & 0xff;
        }
        // blocks open only at slots that are multiples of four
        const unsigned starts = __ballot_sync(FULL, opens);
        __syncwarp();
#pragma unroll
        for (int q = 0; q < 32; q += 4) {
          const float4 fv = *reinterpret_cast<const float4 *>(fr + q);
          const float4 fdv = *reinterpret_cast<const float4 *>(fdr + q);
          const float4 gv = *reinterpret_cast<const float4 *>(gr + q);
          const float4 gdv = *reinterpret_cast<const float4 *>(gdr + q);
          if ((starts >> q) & 1u) open(W.b.sp[q]);
          const float2 f01 = make_float2(fv.x, fv.y), f23 = make_float2(fv.z, fv.w);
          const float2 g01 = make_float2(gv.x, gv.y), g23 = make_float2(gv.z, gv.w);
          ra = fma2(make_float2(fdv.x, fdv.y), g01, fma2(f01, make_float2(gdv.x, gdv.y), ra));
          rb = fma2(make_float2(fdv.z, fdv.w), g23, fma2(f23, make_float2(gdv.z, gdv.w), rb));
          qa = fma2(f01, g01, qa);
          qb = fma2(f23, g23, qb);
        }
        __syncwarp();
      }
      open(-1);
    }
    __syncwarp();
  }
}

// ------------------------------------------------------------------------------ small systems
// Energies, forces and virials of a small system (atoms x members at most SMALL_EVAL_ROWS) in one launch of
// thread-block clusters: the AEV forward, the networks forward (members fused in the first layer) and
// backward to dE/dAEV in FP32 FFMA, and the AEV adjoint.  The atoms are cut into row groups (up to 16 atoms
// of one element, in species order); a cluster owns whole row groups, so every stage of its rows reads only
// what its own CTAs wrote and the stages are separated by cluster barriers (no grid-wide barrier).  Every
// dense layer of a cluster is cut into tasks of (member, row group, 32 or 16 output columns) spread over its
// CTAs, each reducing K across its 8 warps in a fixed order; the last CTA to finish sums the energies in a
// fixed order, so they are deterministic.  A single 128-row tensor-core tile would sit on one SM.
constexpr int SE_WARPS = 8, SE_RG = 16;
constexpr int SE_CL = 16;        // CTAs per cluster (one SM each)
constexpr int SE_MAXCL = 4;      // clusters per launch
constexpr int SE_MAXG = SMALL_BUILD_ATOMS / SE_RG + NE;   // row groups of a system, at most

struct GridBar {
  unsigned count, gen, pad0, pad1;   // CTAs finished (the last one sums the energies); zeroed before a launch
};

// every thread of every CTA of the cluster: arrive (release) and wait (acquire) at the cluster barrier, which
// orders the CTAs' global-memory writes before the stage that reads them
__device__ __forceinline__ void cluster_sync_all() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
__device__ __forceinline__ int cluster_rank() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return (int)r;
}

// the row groups a cluster owns: element, first position in the species-sorted atom list, atoms
struct SmallGroups {
  int n;
  int e[SE_MAXG], base[SE_MAXG], R[SE_MAXG];
};

struct SmallEvalArgs {
  AevFwdArgs fa;
  AevAdjArgs aa;
  int N, NM, M;
  const int32_t *mol_offsets;
  const uint8_t *elem;
  const int32_t *perm;     // atom -> species-sorted row
  const int32_t *meta;     // META_SEG
  const float *W1T, *b1, *W2T, *b2, *W3T, *b3, *w4, *b4, *W3, *W2, *W1;
  float *aev, *h1, *h2, *g3, *g2, *g1, *gaev;   // [N][...] in atom order
  float *ysl;              // [N][M][SE_YCH] output-layer partial sums per third-layer column chunk
  double *E;
  float *F;
  double *virial;
  GridBar *bar;
  DevStatus *st;
};

constexpr int SE_KC = 1024;  // K staged at once (a longer K -- the first layer's input gradient above four
                             // members -- in steps of SE_KC, each waited for)
constexpr int SE_YCH = H3 / 32;   // third-layer column chunks: output-layer partial sums per row and member
struct SmallDense {
  float As[SE_RG][SE_KC];
  float Bs[SE_KC][32];
  float red[SE_WARPS][SE_RG][32];
  float tmp[SE_RG][33];
  float ep_bias[32], ep_w4[32];   // the epilogue's bias and output-layer weights of the chunk
  float ep_aux[SE_RG][32];        // and its CELU' operand rows
  int rows[SE_RG];
};
union SmallShared {
  FwdStage fwd[SE_WARPS];
  AdjStage adj[SE_WARPS];
  SmallDense d;
};

// Task t of a layer over a cluster's row groups: member, element, row group (atoms rows[0..R)), column chunk.
struct SmallTask {
  int m, e, R, chunk;
};
__device__ bool small_task(const SmallGroups &G, const int *srow, int t, int n_chunks, int members, SmallTask &k,
                           int *rows) {
  const int per_m = G.n * n_chunks;
  if (t >= per_m * members) return false;
  k.m = t / per_m;
  const int u = t - k.m * per_m, gi = u / n_chunks;
  k.chunk = u - gi * n_chunks;
  k.e = G.e[gi];
  k.R = G.R[gi];
  if (threadIdx.x < SE_RG) rows[threadIdx.x] = threadIdx.x < k.R ? srow[G.base[gi] + threadIdx.x] : 0;
  return true;
}


// copies of one K chunk [kc0, kc0 + kn) into buffer b: the rows' A values and the 32 columns of B (zeros past
// ncol; every offset is a multiple of four floats, so each copy is 16 aligned bytes)
__device__ __forceinline__ void small_stage(SmallDense &D, const float *A, int lda, int a_off, int R,
                                            const float *B, int ldb, int c0, int ncol, int kc0, int kn, int cw) {
  const int kq = kn / 4;
  for (int q = threadIdx.x; q < R * kq; q += blockDim.x) {
    const int r = q / kq, k4 = (q - r * kq) * 4;
    cp16(&D.As[r][k4], A + (size_t)D.rows[r] * lda + a_off + kc0 + k4);
  }
  const int per = cw / 4;   // 16-byte copies per k row
  for (int q = threadIdx.x; q < kn * per; q += blockDim.x) {
    const int k = q / per, c4 = (q - k * per) * 4;
    if (c0 + c4 < ncol) cp16(&D.Bs[k][c4], B + (size_t)(kc0 + k) * ldb + c0 + c4);
    else *reinterpret_cast<float4 *>(&D.Bs[k][c4]) = make_float4(0.f, 0.f, 0.f, 0.f);
  }
  cp_commit();
}

__device__ __forceinline__ float celu_f(float z) { return z > 0.f ? z : CELU_ALPHA * (__expf(z * CELU_INV_ALPHA) - 1.f); }
// CELU' from the activation h = CELU(z): 1 for z > 0, exp(z / alpha) = 1 + h / alpha otherwise
__device__ __forceinline__ float dcelu_h(float h) { return h > 0.f ? 1.f : fmaf(h, CELU_INV_ALPHA, 1.f); }

// One dense layer over every (member, row group, column chunk) task of the cluster's row groups, spread over
// its CTAs; K in staged chunks, each warp a slice of every chunk, the warps' partial sums added in a fixed
// order.  Chunks are 32 columns (a lane per column), or 16 when that leaves at least half of the cluster's
// CTAs without a task (a lane
// per column and half of the warp's K slice, the halves added by one shuffle); the third layer keeps 32
// (its output-layer partial sums have a slot per 32 columns).
// kind 0: out = CELU(A B + bias); 1: out = (A B) * CELU'(aux); 2: out = A B;
// 3 (third layer): h = CELU(A B + bias), out = w4 CELU'(h) / M, and the output layer's sum of w4 h over the
// chunk's columns into ysl[(row M + m) SE_YCH + chunk]
__device__ void small_layer(const SmallEvalArgs &A, SmallDense &D, const SmallGroups &G, const int *srow, int kind,
                            const float *Ab,
                            int lda, int a_member_off, int K, const float *Bb, long long b_me_stride, int ldb,
                            int ncol, const float *bias, long long bias_me_stride, const float *aux, int ldaux,
                            int aux_member_off, float *out, int ldo, int o_member_off, int members, float *ysl) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int tasks32 = G.n * members * ((ncol + 31) / 32);
  const int cw = (kind != 3 && 2 * tasks32 <= SE_CL) ? 16 : 32;
  const int n_chunks = (ncol + cw - 1) / cw;
  const int nkc = (K + SE_KC - 1) / SE_KC;
  const int col_l = cw == 32 ? lane : (lane & 15), kh = cw == 32 ? 0 : lane >> 4;   // column and K half of the lane
  for (int t = cluster_rank();; t += SE_CL) {
    SmallTask k;
    __syncthreads();
    const bool ok = small_task(G, srow, t, n_chunks, members, k, D.rows);
    __syncthreads();
    if (!ok) break;
    const int c0 = k.chunk * cw;
    const long long me = (long long)(k.m * NE + k.e);
    const float *B = Bb + me * b_me_stride;
    const int a_off = k.m * a_member_off;
    float2 acc2[SE_RG];   // per row: the even-k and odd-k sums, packed
#pragma unroll
    for (int r = 0; r < SE_RG; r++) acc2[r] = make_float2(0.f, 0.f);
    // the epilogue's operands travel with the first operand copies
    if (threadIdx.x < cw / 4) {
      const int c4 = threadIdx.x * 4;
      if (c0 + c4 < ncol) {
        if (kind == 0 || kind == 3) cp16(&D.ep_bias[c4], bias + me * bias_me_stride + c0 + c4);
        if (kind == 3) cp16(&D.ep_w4[c4], A.w4 + me * H3 + c0 + c4);
      }
    }
    if (kind == 1)
      for (int q = threadIdx.x; q < k.R * (cw / 4); q += blockDim.x) {
        const int r = q / (cw / 4), c4 = (q - r * (cw / 4)) * 4;
        if (c0 + c4 < ncol) cp16(&D.ep_aux[r][c4], aux + (size_t)D.rows[r] * ldaux + k.m * aux_member_off + c0 + c4);
      }
    for (int c = 0; c < nkc; c++) {
      const int kc0 = c * SE_KC, kn = min(SE_KC, K - kc0);
      small_stage(D, Ab, lda, a_off, k.R, B, ldb, c0, ncol, kc0, kn, cw);
      cp_wait0();
      __syncthreads();
      // warp w (and K half kh) takes every SE_WARPS-th (2 SE_WARPS-th) group of four k (interleaved: every
      // warp busy for any kn)
      const int kst = cw == 32 ? 4 * SE_WARPS : 8 * SE_WARPS;
      for (int kk = cw == 32 ? 4 * warp : 4 * (2 * warp + kh); kk < kn; kk += kst) {
        const float2 b01 = make_float2(D.Bs[kk][col_l], D.Bs[kk + 1][col_l]);
        const float2 b23 = make_float2(D.Bs[kk + 2][col_l], D.Bs[kk + 3][col_l]);
#pragma unroll
        for (int r = 0; r < SE_RG; r++) {
          if (r < k.R) {
            const float4 a = *reinterpret_cast<const float4 *>(&D.As[r][kk]);
            acc2[r] = fma2(make_float2(a.x, a.y), b01, fma2(make_float2(a.z, a.w), b23, acc2[r]));
          }
        }
      }
      __syncthreads();   // before the buffers are staged again
    }
    float acc[SE_RG];
#pragma unroll
    for (int r = 0; r < SE_RG; r++) acc[r] = acc2[r].x + acc2[r].y;
    if (cw == 16)
#pragma unroll
      for (int r = 0; r < SE_RG; r++) acc[r] += __shfl_xor_sync(FULL, acc[r], 16);
#pragma unroll
    for (int r = 0; r < SE_RG; r++) D.red[warp][r][lane] = acc[r];
    __syncthreads();
    for (int q = threadIdx.x; q < k.R * 32; q += blockDim.x) {
      const int r = q >> 5, l = q & 31, col = l < cw ? c0 + l : ncol;
      float z = 0.f;
#pragma unroll
      for (int w = 0; w < SE_WARPS; w++) z += D.red[w][r][l];   // fixed order
      const int row = D.rows[r];
      float yv = 0.f;
      if (col < ncol) {
        float v;
        if (kind == 0) {
          v = celu_f(z + D.ep_bias[l]);
        } else if (kind == 1) {
          v = z * dcelu_h(D.ep_aux[r][l]);
        } else if (kind == 2) {
          v = z;
        } else {
          const float h = celu_f(z + D.ep_bias[l]), w = D.ep_w4[l];
          v = w * dcelu_h(h) / (float)A.M;
          yv = w * h;
        }
        out[(size_t)row * ldo + k.m * o_member_off + col] = v;
      }
      if (kind == 3) D.tmp[r][l] = yv;
    }
    if (kind == 3) {
      __syncthreads();
      if (threadIdx.x < k.R) {
        float ys = 0.f;
        for (int l = 0; l < 32; l++) ys += D.tmp[threadIdx.x][l];   // fixed order
        ysl[((size_t)D.rows[threadIdx.x] * A.M + k.m) * SE_YCH + k.chunk] = ys;
      }
    }
  }
}

__global__ void __launch_bounds__(SE_WARPS * 32, 1) k_small_eval(SmallEvalArgs A) {
  extern __shared__ __align__(16) unsigned char small_eval_dyn[];
  SmallShared &S = *reinterpret_cast<SmallShared *>(small_eval_dyn);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int M = A.M, N = A.N;
  const int crank = cluster_rank(), cid = (int)blockIdx.x / SE_CL, ncl = (int)gridDim.x / SE_CL;
  // element counts and the atoms in element order (every CTA; from the species order of the list)
  __shared__ int ecount[NE], estart[NE + 1];
  __shared__ int srow[SMALL_BUILD_ATOMS];
  // the row groups of this cluster (groups cid, cid + ncl, ... of the element-major list) and their atoms
  __shared__ SmallGroups G;
  __shared__ int goff[SE_MAXG];   // first position of each owned group in crow
  __shared__ int crow[SMALL_BUILD_ATOMS];
  __shared__ int n_crow, last_cta;
  if (threadIdx.x < NE) ecount[threadIdx.x] = 0;
  __syncthreads();
  for (int i = threadIdx.x; i < N; i += blockDim.x) atomicAdd(&ecount[A.elem[i]], 1);
  __syncthreads();
  if (threadIdx.x == 0) {
    estart[0] = 0;
    for (int e = 0; e < NE; e++) estart[e + 1] = estart[e] + ecount[e];
    int g = 0, n = 0;
    for (int e = 0; e < NE; e++)
      for (int r0 = 0; r0 < ecount[e]; r0 += SE_RG, g++)
        if (g % ncl == cid) {
          G.e[n] = e;
          G.base[n] = estart[e] + r0;
          G.R[n] = min(SE_RG, ecount[e] - r0);
          goff[n] = n == 0 ? 0 : goff[n - 1] + G.R[n - 1];
          n++;
        }
    G.n = n;
    n_crow = n ? goff[n - 1] + G.R[n - 1] : 0;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    const int e = A.elem[i];
    srow[estart[e] + A.perm[i] - A.meta[META_SEG + e]] = i;
  }
  __syncthreads();
  for (int q = 0; q < G.n; q++)
    for (int r = threadIdx.x; r < G.R[q]; r += blockDim.x) crow[goff[q] + r] = srow[G.base[q] + r];
  __syncthreads();
  // the cluster's warps over its atoms: a row per warp, or (fewer rows than warps) up to eight warps per row
  const int wg = crank * SE_WARPS + warp, nw = SE_CL * SE_WARPS;
  const int Kw = min(8, max(1, nw / max(n_crow, 1)));
  // AEV rows (atom order)
  if (Kw > 1) aev_forward_parts<float>(A.fa, S.fwd[warp], wg, nw, Kw, crow, n_crow);
  else aev_forward_rows<float>(A.fa, S.fwd[warp], wg, nw, crow, n_crow);
  cluster_sync_all();
  SmallDense &D = S.d;
  const int MH1 = M * H1;
  // first layer, all members fused: h1 = CELU(aev W1^T + b1), [N][M 256]
  small_layer(A, D, G, srow, 0, A.aev, NAEV, 0, NAEV, A.W1T, (long long)NAEV * MH1, MH1, MH1, A.b1, MH1, nullptr, 0, 0,
              A.h1, MH1, 0, 1, nullptr);
  cluster_sync_all();
  // second layer per member: h2 = CELU(h1_m W2^T + b2), [N][M 192]
  small_layer(A, D, G, srow, 0, A.h1, MH1, H1, H1, A.W2T, (long long)H1 * H2, H2, H2, A.b2, H2, nullptr, 0, 0, A.h2, M * H2,
              H2, M, nullptr);
  cluster_sync_all();
  // third layer per member: h3 = CELU(h2_m W3^T + b3) -> g3 = (1/M) w4 CELU'(z3) and the output layer's
  // partial sums per column chunk (fixed slots, added in a fixed order with the energies)
  small_layer(A, D, G, srow, 3, A.h2, M * H2, H2, H2, A.W3T, (long long)H2 * H3, H3, H3, A.b3, H3, nullptr, 0, 0, A.g3,
              M * H3, H3, M, A.ysl);
  cluster_sync_all();
  // third layer's input gradient: g2 = (g3 W3) * CELU'(h2)
  small_layer(A, D, G, srow, 1, A.g3, M * H3, H3, H3, A.W3, (long long)H3 * H2, H2, H2, nullptr, 0, A.h2, M * H2, H2, A.g2,
              M * H2, H2, M, nullptr);
  cluster_sync_all();
  // second layer's: g1 = (g2 W2) * CELU'(h1)
  small_layer(A, D, G, srow, 1, A.g2, M * H2, H2, H2, A.W2, (long long)H2 * H1, H1, H1, nullptr, 0, A.h1, MH1, H1, A.g1,
              MH1, H1, M, nullptr);
  cluster_sync_all();
  // first layer's, summed over the members: dE/dAEV = g1 W1 (K = M 256 through the member-concatenated W1)
  small_layer(A, D, G, srow, 2, A.g1, MH1, 0, MH1, A.W1, (long long)MH1 * NAEV, NAEV, NAEV, nullptr, 0, nullptr, 0, 0,
              A.gaev, NAEV, 0, 1, nullptr);
  cluster_sync_all();
  // forces and virials of the cluster's atoms (F and the virials were zeroed before the launch)
  aev_adjoint_rows(A.aa, S.adj[warp], wg, nw, Kw, crow, n_crow);
  // the energies, by the last CTA to finish (every CTA's output-layer sums are written by then): a warp per
  // structure, lanes over its atoms, then a shuffle tree (a fixed order)
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    last_cta = atomicAdd(&A.bar->count, 1u) == gridDim.x - 1;
    __threadfence();
  }
  __syncthreads();
  if (!last_cta) return;
  for (int m = warp; m < A.NM; m += SE_WARPS) {
    const int a0 = max(A.mol_offsets[m], 0), a1 = min(A.mol_offsets[m + 1], N);
    double e = 0.0;
    for (int i = a0 + lane; i < a1; i += 32) {
      const int el = A.elem[i];
      double yi = 0.0;
      for (int q = 0; q < M; q++) {
        float yq = A.b4[q * NE + el];
        for (int c = 0; c < SE_YCH; c++) yq += __ldcg(&A.ysl[((size_t)i * M + q) * SE_YCH + c]);
        yi += (double)yq;
      }
      e += yi / (double)M;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) e += __shfl_xor_sync(0xffffffffu, e, o);
    if (lane != 0) continue;
    A.E[m] = e;
    if (!isfinite(e)) post_status(A.st, FNN_E_NONFINITE, -(long long)(m + 1));
  }
}

// before each evaluation: the finish count, the forces and the virials, which the clusters accumulate into
__global__ void k_small_zero(GridBar *bar, float *F, int nf, double *virial, int nv) {
  if (blockIdx.x == 0 && threadIdx.x == 0) bar->count = 0;
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < nf; q += gridDim.x * blockDim.x) F[q] = 0.f;
  if (virial)
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < nv; q += gridDim.x * blockDim.x) virial[q] = 0.0;
}

static StageArgs stage_args(const fnn_system *sys, const fnn_nlist *nl) {
  StageArgs s;
  s.cap = nl->capacity;
  s.sorted_upto = PAIR_STRIDE;
  s.pos = reinterpret_cast<const float4 *>(sys->pos);
  s.row_ptr = nl->row_ptr;
  s.nbr = nl->nbr;
  s.shift = nl->shift;
  s.elem = nl->elem;
  s.atom_mol = nl->atom_mol;
  s.grid = nl->grid;
  return s;
}

// one wave of resident blocks (per_sm per SM, the kernel's launch bound) walking the rows
static int aev_grid(fnn_ctx *ctx, int64_t rows, int per_sm, int warps = AEV_WARPS) {
  int64_t need = (rows + warps - 1) / warps;
  int64_t cap = (int64_t)ctx->num_sms * per_sm;
  if (need > cap) need = cap;
  return need < 1 ? 1 : (int)need;
}

fnn_status launch_aev_forward(fnn_ctx *ctx, const fnn_system *sys, const fnn_nlist *nl, float *out,
                              const int32_t *inv, cudaStream_t s) {
  AevFwdArgs a;
  a.sa = stage_args(sys, nl);
  a.P = ctx->aev;
  a.out = out;
  a.out_lo = nullptr;
  a.out_inv = 1.f;
  a.inv = inv;
  a.meta = nl->meta;
  a.n_atoms = sys->n_atoms;
  a.st = ctx->status;
  int64_t rows = inv ? nl->pad_cap : sys->n_atoms;
  if (rows == 0) return FNN_OK;
  {
    FNN_KERNEL(ctx, "aev_forward", s);
    k_aev_forward<float><<<aev_grid(ctx, rows * 8, AEV_FWD_BLOCKS), AEV_WARPS * 32, 0, s>>>(a);
  }
  return check_launch(ctx, "aev_forward");
}

fnn_status launch_aev_forward_bf16(fnn_ctx *ctx, const fnn_system *sys, const fnn_nlist *nl, __nv_bfloat16 *out,
                                   __nv_bfloat16 *out_lo, const int32_t *inv, cudaStream_t s) {
  AevFwdArgs a;
  a.sa = stage_args(sys, nl);
  a.P = ctx->aev;
  a.out = reinterpret_cast<float *>(out);
  a.out_lo = out_lo;
  a.out_inv = 1.f;
  a.inv = inv;
  a.meta = nl->meta;
  a.n_atoms = sys->n_atoms;
  a.st = ctx->status;
  int64_t rows = inv ? nl->pad_cap : sys->n_atoms;
  if (rows == 0) return FNN_OK;
  {
    FNN_KERNEL(ctx, out_lo ? "aev_forward_x3" : "aev_forward_bf16", s);
    k_aev_forward<__nv_bfloat16><<<aev_grid(ctx, rows * 8, AEV_FWD_BLOCKS), AEV_WARPS * 32, 0, s>>>(a);
  }
  return check_launch(ctx, "aev_forward_bf16");
}

fnn_status launch_aev_l1_bf16(fnn_ctx *ctx, const fnn_system *sys, const fnn_nlist *nl, const CUtensorMap *mW1,
                              const float *b1cat, __nv_bfloat16 *h1, int M, cudaStream_t s) {
  FuseArgs a;
  a.aev.sa = stage_args(sys, nl);
  a.aev.P = ctx->aev;
  a.aev.out = nullptr;
  a.aev.out_lo = nullptr;
  a.aev.out_inv = 1.f;
  a.aev.inv = nl->inv;
  a.aev.meta = nl->meta;
  a.aev.n_atoms = sys->n_atoms;
  a.aev.st = ctx->status;
  a.tile_elem = nl->tile_elem;
  a.rows_cap = nl->pad_cap;
  a.bias = b1cat;
  a.h1 = h1;
  a.M = M;
  const long long tiles = nl->pad_cap / FUSE_ROWS;
  if (tiles == 0) return FNN_OK;
  static bool attr_set = false;
  if (!attr_set) {
    FNN_CUDA_TRY(ctx, cudaFuncSetAttribute(k_aev_l1, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fuse_smem_bytes()));
    attr_set = true;
  }
  {
    FNN_KERNEL(ctx, "aev_l1_bf16", s);
    k_aev_l1<<<(unsigned)(tiles < ctx->num_sms ? tiles : ctx->num_sms), FUSE_THREADS, fuse_smem_bytes(), s>>>(*mW1, a);
  }
  return check_launch(ctx, "aev_l1_bf16");
}

fnn_status launch_aev_forward_fp8(fnn_ctx *ctx, const fnn_system *sys, const fnn_nlist *nl, uint8_t *out,
                                  float out_inv, const int32_t *inv, cudaStream_t s) {
  AevFwdArgs a;
  a.sa = stage_args(sys, nl);
  a.P = ctx->aev;
  a.out = reinterpret_cast<float *>(out);
  a.out_lo = nullptr;
  a.out_inv = out_inv;
  a.inv = inv;
  a.meta = nl->meta;
  a.n_atoms = sys->n_atoms;
  a.st = ctx->status;
  int64_t rows = inv ? nl->pad_cap : sys->n_atoms;
  if (rows == 0) return FNN_OK;
  {
    FNN_KERNEL(ctx, "aev_forward_fp8", s);
    k_aev_forward<__nv_fp8_e4m3><<<aev_grid(ctx, rows * 8, AEV_FWD_BLOCKS), AEV_WARPS * 32, 0, s>>>(a);
  }
  return check_launch(ctx, "aev_forward_fp8");
}

fnn_status launch_aev_adjoint(fnn_ctx *ctx, const fnn_system *sys, const fnn_nlist *nl, const float *gaev,
                              const int32_t *inv, float *F, double *virial, cudaStream_t s) {
  AevAdjArgs a;
  a.sa = stage_args(sys, nl);
  a.P = ctx->aev;
  a.gaev = gaev;
  a.inv = inv;
  a.meta = nl->meta;
  a.n_atoms = sys->n_atoms;
  a.F = F;
  a.virial = virial;
  a.st = ctx->status;
  int64_t rows = inv ? nl->pad_cap : sys->n_atoms;
  if (rows == 0) return FNN_OK;
  {
    FNN_KERNEL(ctx, "aev_adjoint", s);
    k_aev_adjoint<<<aev_grid(ctx, rows, AEV_ADJ_BLOCKS, ADJ_WARPS), ADJ_WARPS * 32, 0, s>>>(a);
  }
  return check_launch(ctx, "aev_adjoint");
}

template <typename OutT>
static fnn_status tangent(fnn_ctx *ctx, const fnn_system *sys, const fnn_nlist *nl, const float *V, OutT *out,
                          __nv_bfloat16 *out_fwd, const int32_t *inv, cudaStream_t s) {
  AevTanArgs a;
  a.sa = stage_args(sys, nl);
  a.P = ctx->aev;
  a.V = V;
  a.out = out;
  a.out_fwd = out_fwd;
  a.inv = inv;
  a.meta = nl->meta;
  a.n_atoms = sys->n_atoms;
  a.st = ctx->status;
  int64_t rows = inv ? nl->pad_cap : sys->n_atoms;
  if (rows == 0) return FNN_OK;
  {
    FNN_KERNEL(ctx, "aev_tangent", s);
    k_aev_tangent<OutT><<<aev_grid(ctx, rows, TAN_BLOCKS), TAN_WARPS * 32, 0, s>>>(a);
  }
  return check_launch(ctx, "aev_tangent");
}

fnn_status launch_aev_tangent(fnn_ctx *ctx, const fnn_system *sys, const fnn_nlist *nl, const float *V, float *out,
                              const int32_t *inv, cudaStream_t s) {
  return tangent<float>(ctx, sys, nl, V, out, nullptr, inv, s);
}
fnn_status launch_aev_tangent_bf16(fnn_ctx *ctx, const fnn_system *sys, const fnn_nlist *nl, const float *V,
                                   __nv_bfloat16 *out, __nv_bfloat16 *out_fwd, const int32_t *inv, cudaStream_t s) {
  return tangent<__nv_bfloat16>(ctx, sys, nl, V, out, out_fwd, inv, s);
}


fnn_status launch_small_eval(fnn_ctx *ctx, const fnn_system *sys, const fnn_nlist *nl, double *E, float *F,
                             double *virial, cudaStream_t s) {
  const int N = sys->n_atoms, M = ctx->cfg.n_members;
  // the barrier word, then the output-layer partial sums (atoms x members x chunks at most SMALL_EVAL_ROWS x 5)
  if (!ctx->grid_bar) FNN_CUDA_TRY(ctx, cudaMalloc(&ctx->grid_bar, 256 + (size_t)SMALL_EVAL_ROWS * SE_YCH * sizeof(float)));
  const size_t dyn = sizeof(SmallShared);
  cudaLaunchConfig_t cfg{};
  cfg.blockDim = dim3(SE_WARPS * 32);
  cfg.dynamicSmemBytes = dyn;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = SE_CL;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  static bool attr_set = false;
  static int max_clusters = 0;
  if (!attr_set) {
    FNN_CUDA_TRY(ctx, cudaFuncSetAttribute(k_small_eval, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn));
    FNN_CUDA_TRY(ctx, cudaFuncSetAttribute(k_small_eval, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
    cfg.gridDim = dim3(SE_CL * SE_MAXCL);
    FNN_CUDA_TRY(ctx, cudaOccupancyMaxActiveClusters(&max_clusters, k_small_eval, &cfg));
    attr_set = true;
  }
  if (max_clusters < 1) {
    ctx->last_error = "small-system kernel: no cluster of 16 CTAs fits on the device";
    return FNN_E_CUDA;
  }
  Workspace &ws = ctx->ws;
  const DeviceWeights &w = ctx->w;
  SmallEvalArgs a{};
  a.fa.sa = stage_args(sys, nl);
  a.fa.P = ctx->aev;
  a.fa.out = ws.aev;
  a.fa.out_lo = nullptr;
  a.fa.out_inv = 1.f;
  a.fa.inv = nullptr;
  a.fa.meta = nl->meta;
  a.fa.n_atoms = N;
  a.fa.st = ctx->status;
  a.aa.sa = a.fa.sa;
  a.aa.P = ctx->aev;
  a.aa.gaev = ws.gaev;
  a.aa.inv = nullptr;
  a.aa.meta = nl->meta;
  a.aa.n_atoms = N;
  a.aa.F = F;
  a.aa.virial = virial;
  a.aa.st = ctx->status;
  a.N = N;
  a.NM = sys->n_mol;
  a.M = M;
  a.mol_offsets = sys->mol_offsets;
  a.elem = nl->elem;
  a.perm = nl->perm;
  a.meta = nl->meta;
  a.W1T = w.W1Tcat;
  a.b1 = w.b1cat;
  a.W2T = w.W2T;
  a.b2 = w.b2;
  a.W3T = w.W3T;
  a.b3 = w.b3;
  a.w4 = w.w4;
  a.b4 = w.b4;
  a.W3 = w.W3;
  a.W2 = w.W2;
  a.W1 = w.W1cat;
  a.aev = ws.aev;
  a.h1 = ws.h1;
  a.h2 = ws.h2;
  a.g3 = ws.g3;
  a.g2 = ws.g2;
  a.g1 = ws.g1;
  a.gaev = ws.gaev;
  a.ysl = reinterpret_cast<float *>(reinterpret_cast<char *>(ctx->grid_bar) + 256);
  a.E = E;
  a.F = F;
  a.virial = virial;
  a.bar = reinterpret_cast<GridBar *>(ctx->grid_bar);
  a.st = ctx->status;
  // clusters: at most one per row group (an upper bound: ceil(N / 16) + 7), SE_MAXCL, and the clusters that fit
  // at once (they never wait on one another, so fewer would still finish)
  const int row_groups = (N + SE_RG - 1) / SE_RG + NE;
  int ncl = row_groups < SE_MAXCL ? row_groups : SE_MAXCL;
  if (ncl > max_clusters) ncl = max_clusters;
  {
    FNN_KERNEL(ctx, "small_zero", s);
    k_small_zero<<<1, 256, 0, s>>>(a.bar, F, 3 * N, virial, 9 * sys->n_mol);
  }
  cfg.gridDim = dim3(SE_CL * ncl);
  {
    FNN_KERNEL(ctx, "small_eval", s);
    FNN_CUDA_TRY(ctx, cudaLaunchKernelEx(&cfg, k_small_eval, a));
  }
  (void)M;
  return check_launch(ctx, "small_eval");
}

}  // namespace fnn
