// Cell-list neighbour search (section II.A graph semantics; cell lists per section V.E) and the
// species-sorted atom order used by the networks.
//
// Pipeline (one stream, no host synchronisation):
//   k_check_cover   offsets start at 0, end at N, never decrease
//   k_atom_setup    per atom: structure (binary search of the offsets), species, bounding boxes
//   k_mol_grid      per structure: validate cell, cell-grid geometry, predicate band
//                   (the allocation-free entry point keeps k_mol_setup: a block per structure)
//   scan            structure cell counts -> first global cell of each structure
//   k_bin           per atom: cell index, histogram (atomics)
//   scan            cell counts -> cell starts (counting sort)
//   k_scatter       atoms into cells; k_sort_cells orders each cell by atom index (determinism)
//   k_pairs_stage   block per cell: its 27-cell stencil staged in shared memory, a warp per centre atom:
//                   predicate, ballot + popc compaction into the atom's 128-entry staging slot, its count
//   scan            counts -> CSR row pointers
//   k_pairs_compact staged rows copied into the CSR list (rows longer than the slot: traversed again)
//   (the allocation-free entry point keeps the two-traversal form: k_pairs<COUNT>, scan, k_pairs<FILL>)
//   k_elem_*        stable counting sort of atoms by element into 128-row padded segments
#include <cfloat>

#include "fnn_internal.cuh"

namespace fnn {

static constexpr unsigned FULL = 0xffffffffu;

// ------------------------------------------------------------------------------------------ scan
__device__ __forceinline__ int warp_incl_scan(int v) {
  int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int t = __shfl_up_sync(FULL, v, o);
    if (lane >= o) v += t;
  }
  return v;
}

// exclusive scan across a block of NT threads; *total receives the block sum (all threads)
template <int NT>
__device__ __forceinline__ int block_excl_scan(int v, int *total) {
  __shared__ int warp_sums[NT / 32];
  __shared__ int tot;
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int inc = warp_incl_scan(v);
  if (lane == 31) warp_sums[w] = inc;
  __syncthreads();
  if (w == 0) {
    int s = lane < NT / 32 ? warp_sums[lane] : 0;
    int si = warp_incl_scan(s);
    if (lane < NT / 32) warp_sums[lane] = si - s;
    if (lane == NT / 32 - 1) tot = si;
  }
  __syncthreads();
  int r = inc - v + warp_sums[w];
  *total = tot;
  __syncthreads();
  return r;
}

constexpr int SCAN_NT = 512, SCAN_ITEMS = 4, SCAN_TILE = SCAN_NT * SCAN_ITEMS;

__global__ void k_scan_tiles(int32_t *data, int64_t n, int32_t *tile_sums) {
  int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
  int v[SCAN_ITEMS];
  int s = 0;
#pragma unroll
  for (int k = 0; k < SCAN_ITEMS; k++) {
    v[k] = base + k < n ? data[base + k] : 0;
    s += v[k];
  }
  int tot;
  int ex = block_excl_scan<SCAN_NT>(s, &tot);
#pragma unroll
  for (int k = 0; k < SCAN_ITEMS; k++) {
    if (base + k < n) data[base + k] = ex;
    ex += v[k];
  }
  if (threadIdx.x == 0) tile_sums[blockIdx.x] = tot;
}

// single block: exclusive scan of the tile sums in chunks, total to *total_dev
__global__ void k_scan_top(int32_t *tile_sums, int64_t nt, int32_t *total_dev) {
  int carry = 0;
  for (int64_t c = 0; c < nt; c += SCAN_NT) {
    int64_t k = c + threadIdx.x;
    int v = k < nt ? tile_sums[k] : 0;
    int tot;
    int ex = block_excl_scan<SCAN_NT>(v, &tot);
    if (k < nt) tile_sums[k] = ex + carry;
    carry += tot;
  }
  if (threadIdx.x == 0 && total_dev) *total_dev = carry;
}

__global__ void k_scan_add(int32_t *data, int64_t n, const int32_t *tile_sums) {
  int add = tile_sums[blockIdx.x];
  int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
  for (int k = threadIdx.x; k < SCAN_TILE; k += SCAN_NT)
    if (base + k < n) data[base + k] += add;
}

// one block for a short array: chunks of SCAN_TILE with a running carry (see exclusive_scan for the arguments)
__global__ void k_scan_small(const int32_t *in, int32_t *out, int32_t *out2, int64_t n, int32_t *total_dev,
                             int64_t cap, DevStatus *st) {
  int carry = 0;
  for (int64_t c = 0; c < n; c += SCAN_TILE) {
    const int64_t base = c + (int64_t)threadIdx.x * SCAN_ITEMS;
    int v[SCAN_ITEMS];
    int sum = 0;
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; k++) {
      v[k] = base + k < n ? in[base + k] : 0;
      sum += v[k];
    }
    int tot;
    int ex = block_excl_scan<SCAN_NT>(sum, &tot) + carry;
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; k++) {
      if (base + k < n) {
        out[base + k] = ex;
        if (out2) out2[base + k] = ex;
      }
      ex += v[k];
    }
    carry += tot;
  }
  if (threadIdx.x == 0) {
    if (total_dev) *total_dev = carry;
    if (cap >= 0 && carry > cap) post_status(st, FNN_E_CAPACITY, carry);
  }
}

// Single-pass scan of long arrays (decoupled look-back, Merrill and Garland 2016).  Blocks take tiles
// in the order they start (a ticket), so every tile a block waits on belongs to a block that is
// already running.  Each tile publishes one 64-bit word per tile: flag (1 = its own sum, 2 = sum of
// everything up to and including it) << 32 | value.  The scratch holds the ticket, a pad word and the
// tile words, and must be zero at launch.  n_dev, when given, bounds the scanned length at run time to
// min(n_max, *n_dev + 1) (a count known only on the device); blocks past it return at once.
constexpr long long LOOKBACK_LIMIT = 2000000000LL;   // clock64 cycles (about a second) per wait

__global__ void __launch_bounds__(SCAN_NT) k_scan_single_pass(const int32_t *in, int32_t *out, int32_t *out2,
                                                              int64_t n_max, const int32_t *n_dev,
                                                              int32_t *total_dev, int64_t cap, int32_t *scratch,
                                                              DevStatus *st, int withhold_first = 0) {
  __shared__ int tile_s, prefix_s;
  unsigned *ticket = reinterpret_cast<unsigned *>(scratch);
  unsigned long long *word = reinterpret_cast<unsigned long long *>(scratch + 2);
  if (threadIdx.x == 0) tile_s = (int)atomicAdd(ticket, 1u);
  __syncthreads();
  const int t = tile_s;
  const int64_t n = n_dev ? min(n_max, (int64_t)*n_dev + 1) : n_max;
  const int64_t base0 = (int64_t)t * SCAN_TILE;
  if (base0 >= n) return;   // uniform over the block
  const int64_t base = base0 + (int64_t)threadIdx.x * SCAN_ITEMS;
  int v[SCAN_ITEMS];
  int sum = 0;
#pragma unroll
  for (int k = 0; k < SCAN_ITEMS; k++) {
    v[k] = base + k < n ? in[base + k] : 0;
    sum += v[k];
  }
  int agg;
  int ex = block_excl_scan<SCAN_NT>(sum, &agg);
  if (threadIdx.x < 32) {   // warp 0: publish, look back, publish the inclusive prefix
    const int lane = threadIdx.x;
    int prefix = 0;
    if (t > 0) {
      if (lane == 0) atomicExch(&word[t], (1ull << 32) | (unsigned)agg);
      int j = t - 1;   // nearest predecessor not yet accounted for
      bool done = false;
      while (!done) {
        const int idx = j - lane;
        unsigned long long w = 2ull << 32;   // before tile 0: an inclusive zero
        if (idx >= 0) {
          volatile unsigned long long *pw = word + idx;
          w = *pw;
          if ((w >> 32) == 0) {
            const long long t0 = clock64();
            while (((w = *pw) >> 32) == 0)
              if (clock64() - t0 > LOOKBACK_LIMIT) {
                post_status(st, FNN_E_TIMEOUT, t);
                w = 2ull << 32;
                break;
              }
          }
        }
        const unsigned incl = __ballot_sync(FULL, (w >> 32) == 2);
        const int stop = incl ? __ffs(incl) - 1 : 31;   // lanes 0..stop contribute
        int val = lane <= stop ? (int)(unsigned)(w & 0xffffffffull) : 0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) val += __shfl_xor_sync(FULL, val, o);
        prefix += val;
        done = incl != 0;
        j -= 32;
      }
    }
    if (lane == 0) {
      // (withhold_first: the self-test of the bounded wait; tile 0 never publishes, so its successors'
      // waits run out)
      if (!(withhold_first && t == 0)) atomicExch(&word[t], (2ull << 32) | (unsigned)(prefix + agg));
      prefix_s = prefix;
      if (base0 + SCAN_TILE >= n) {   // the last tile
        if (total_dev) *total_dev = prefix + agg;
        if (cap >= 0 && prefix + agg > cap) post_status(st, FNN_E_CAPACITY, prefix + agg);
      }
    }
  }
  __syncthreads();
  ex += prefix_s;
#pragma unroll
  for (int k = 0; k < SCAN_ITEMS; k++) {
    if (base + k < n) {
      out[base + k] = ex;
      if (out2) out2[base + k] = ex;
    }
    ex += v[k];
  }
}

int64_t scan_tmp_needed(int64_t n) { return 2 * ((n + SCAN_TILE - 1) / SCAN_TILE) + 2; }

// out[k] = in[0] + ... + in[k-1] for k < n (in and out may be the same array; so may out2, a second copy),
// the total to *total_dev, and FNN_E_CAPACITY posted when the total exceeds cap (cap >= 0).  n_dev, when
// given, bounds n at run time to min(n, *n_dev + 1).  tmp (tmp_len int32) is the single-pass scratch; with
// zeroed set the caller has cleared it since its last use (no memset node).
fnn_status exclusive_scan(fnn_ctx *ctx, const int32_t *in, int32_t *out, int64_t n, int32_t *total_dev, int32_t *tmp,
                          int64_t tmp_len, cudaStream_t s, const int32_t *n_dev, int32_t *out2, int64_t cap,
                          bool zeroed) {
  if (n <= 0) return FNN_OK;
  if (n <= 2 * SCAN_TILE && !n_dev) {   // one block for short arrays (structure and small cell counts)
    FNN_KERNEL(ctx, "scan_small", s);
    k_scan_small<<<1, SCAN_NT, 0, s>>>(in, out, out2, n, total_dev, cap, ctx->status);
    return check_launch(ctx, "exclusive_scan");
  }
  const int64_t nt = (n + SCAN_TILE - 1) / SCAN_TILE;
  if (2 * nt + 2 > tmp_len) {
    ctx->last_error = "scan scratch too small";
    return FNN_E_INVALID;
  }
  if (!zeroed) FNN_CUDA_TRY(ctx, cudaMemsetAsync(tmp, 0, (size_t)(2 * nt + 2) * sizeof(int32_t), s));
  FNN_KERNEL(ctx, "scan", s);
  k_scan_single_pass<<<(unsigned)nt, SCAN_NT, 0, s>>>(in, out, out2, n, n_dev, total_dev, cap, tmp, ctx->status);
  return check_launch(ctx, "exclusive_scan");
}

// Self-test of the look-back's bounded wait (fnn_selftest_lookback): a scan of SELFTEST_TILES tiles of
// ones in a library-owned buffer, optionally with tile 0's publication withheld.  Nothing reads the
// result but k_selftest_check, which posts FNN_E_INVALID when a scan that was not withheld is wrong.
constexpr int SELFTEST_TILES = 3;
__global__ void k_selftest_fill(int32_t *data, int64_t n, int32_t *scratch, int64_t n_scratch) {
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
    data[k] = 1;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n_scratch;
       k += (int64_t)gridDim.x * blockDim.x)
    scratch[k] = 0;
}
__global__ void k_selftest_check(const int32_t *data, int64_t n, DevStatus *st) {
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
    if (data[k] != (int32_t)k) post_status(st, FNN_E_INVALID, k);
}

// ------------------------------------------------------------------------------------- structures
// offsets must start at 0, end at N and never decrease: otherwise some atom has no structure, or
// structures overlap.  The verdict is global: the first block checks every offset and writes bad[0]
// (0 or 1) once, so the later setup kernels can drop every structure of an inconsistent batch (per
// structure checks alone would let overlapping structures claim more cells than the bound allows).
// The other blocks reset the per-structure bounding boxes, when given, to empty, and clear, when given,
// meta (except META_BAD), the structure cell counts and the scan scratch.
__global__ void k_check_cover(fnn_system sys, DevStatus *st, float *bbox, int32_t *meta, int32_t *mol_cells,
                              int32_t *scratch, int64_t n_scratch, int32_t *bad) {
  if (blockIdx.x == 0) {
    int any = 0;
    for (int m = threadIdx.x; m <= sys.n_mol; m += blockDim.x) {
      const int a = sys.mol_offsets[m];
      bool ok = (m == 0) ? a == 0 : (a >= sys.mol_offsets[m - 1]);
      if (m == sys.n_mol) ok = ok && a == sys.n_atoms;
      if (!ok) {
        post_status(st, FNN_E_INVALID, m);
        any = 1;
      }
    }
    any = __syncthreads_or(any);
    if (threadIdx.x == 0) *bad = any;
  }
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x, ng = (int64_t)gridDim.x * blockDim.x;
  if (meta)
    for (int64_t k = g; k < META_LEN; k += ng)
      if (meta + k != bad) meta[k] = 0;
  if (scratch)
    for (int64_t k = g; k < n_scratch; k += ng) scratch[k] = 0;
  for (int m = blockIdx.x * blockDim.x + threadIdx.x; m <= sys.n_mol; m += gridDim.x * blockDim.x) {
    if (mol_cells) mol_cells[m] = 0;
    if (bbox && m < sys.n_mol)
      for (int a3 = 0; a3 < 3; a3++) {
        bbox[6 * (size_t)m + a3] = __int_as_float(0x7f800000);        // +inf
        bbox[6 * (size_t)m + 3 + a3] = __int_as_float((int)0xff800000);   // -inf
      }
  }
}

// float min / max through integer atomics (valid for finite values and the +-inf initial bounds)
__device__ __forceinline__ void atomic_fmin(float *a, float v) {
  if (v >= 0.f)
    atomicMin(reinterpret_cast<int *>(a), __float_as_int(v));
  else
    atomicMax(reinterpret_cast<unsigned *>(a), __float_as_uint(v));
}
__device__ __forceinline__ void atomic_fmax(float *a, float v) {
  if (v >= 0.f)
    atomicMax(reinterpret_cast<int *>(a), __float_as_int(v));
  else
    atomicMin(reinterpret_cast<unsigned *>(a), __float_as_uint(v));
}

// Per atom, all structures at once: its structure (binary search of the offsets), element, checks, and
// the structure's bounding box (a warp whose atoms share one structure reduces before its atomics).
// (also writes atom_mol = -1 and element 0 for an atom outside every structure, and zeroes counts [N+1])
__global__ void k_atom_setup(fnn_system sys, int32_t *atom_mol, uint8_t *elem, float *bbox, int32_t *counts,
                             DevStatus *st, const int32_t *bad) {
  const float4 *pos = reinterpret_cast<const float4 *>(sys.pos);
  const int lane = threadIdx.x & 31;
  const bool drop = *bad != 0;   // inconsistent offsets: no atom belongs to a structure
  if (counts && blockIdx.x == 0 && threadIdx.x == 0) counts[sys.n_atoms] = 0;
  for (int i0 = blockIdx.x * blockDim.x; i0 < sys.n_atoms; i0 += gridDim.x * blockDim.x) {
    const int i = i0 + threadIdx.x;
    int m = -1;
    float4 p = make_float4(0.f, 0.f, 0.f, 0.f);
    if (i < sys.n_atoms) {
      if (counts) counts[i] = 0;
      int lo = 0, hi = sys.n_mol;   // last m with offsets[m] <= i
      while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (sys.mol_offsets[mid] <= i) lo = mid; else hi = mid;
      }
      if (!drop && sys.mol_offsets[lo] <= i && i < sys.mol_offsets[lo + 1]) m = lo;
      if (m < 0) {
        atom_mol[i] = -1;
        elem[i] = 0;
      } else {
        atom_mol[i] = m;
        int e = element_of(sys.Z[i]);
        if (e < 0) {
          post_status(st, FNN_E_SPECIES, i);
          e = 0;
        }
        elem[i] = (uint8_t)e;
        p = pos[i];
        if (!isfinite(p.x) || !isfinite(p.y) || !isfinite(p.z)) post_status(st, FNN_E_NONFINITE, i);
      }
    }
    const int m0 = __shfl_sync(FULL, m, 0);
    if (__all_sync(FULL, m == m0)) {
      if (m0 < 0) continue;
      float v[6] = {p.x, p.y, p.z, p.x, p.y, p.z};
#pragma unroll
      for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int a = 0; a < 3; a++) {
          v[a] = fminf(v[a], __shfl_xor_sync(FULL, v[a], o));
          v[3 + a] = fmaxf(v[3 + a], __shfl_xor_sync(FULL, v[3 + a], o));
        }
      if (lane == 0)
        for (int a = 0; a < 3; a++) {
          atomic_fmin(&bbox[6 * (size_t)m0 + a], v[a]);
          atomic_fmax(&bbox[6 * (size_t)m0 + 3 + a], v[3 + a]);
        }
    } else if (m >= 0) {
      atomic_fmin(&bbox[6 * (size_t)m], p.x);
      atomic_fmin(&bbox[6 * (size_t)m + 1], p.y);
      atomic_fmin(&bbox[6 * (size_t)m + 2], p.z);
      atomic_fmax(&bbox[6 * (size_t)m + 3], p.x);
      atomic_fmax(&bbox[6 * (size_t)m + 4], p.y);
      atomic_fmax(&bbox[6 * (size_t)m + 5], p.z);
    }
  }
}

__device__ MolGrid make_grid(const fnn_system &sys, int m, int n, int pbc, float bb[6], double R, DevStatus *st,
                             int *cells);

// Per structure: offsets check, then the grid from its bounding box
__global__ void k_mol_grid(fnn_system sys, const float *bbox, MolGrid *grid, int32_t *mol_cells, double R,
                           DevStatus *st, const int32_t *bad) {
  const bool drop = *bad != 0;   // inconsistent offsets (posted by k_check_cover): every structure empty
  for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < sys.n_mol; m += gridDim.x * blockDim.x) {
    const int a0 = sys.mol_offsets[m], a1 = sys.mol_offsets[m + 1];
    if (drop || a0 < 0 || a1 < a0 || a1 > sys.n_atoms) {
      post_status(st, FNN_E_INVALID, m);
      grid[m] = MolGrid{0, 0, 0, 0, 0, 0, 0, 0, 0, 1, 1, 1, 0, 0};
      mol_cells[m] = 1;
      continue;
    }
    const int pbc = sys.pbc ? (sys.pbc[m] != 0) : 0;
    float bb[6];
    for (int a = 0; a < 6; a++) bb[a] = bbox[6 * (size_t)m + a];
    int cells;
    grid[m] = make_grid(sys, m, a1 - a0, pbc, bb, R, st, &cells);
    mol_cells[m] = cells;
  }
}

// Cell grid, image data and predicate band of structure m with n atoms and bounding box bb (min xyz, max
// xyz); posts FNN_E_CELL for a cell the minimum image cannot serve.
__device__ MolGrid make_grid(const fnn_system &sys, int m, int n, int pbc, float bb[6], double R, DevStatus *st,
                             int *cells) {
  MolGrid g{};
  double edge = R * (1.0 + 1e-4);   // cells at least this wide: fp32 binning error stays far below the margin
  double ext[3];
  g.pbc = pbc;
  if (pbc) {
    const float *c = sys.cell + 9 * (size_t)m;
    bool ortho = c[1] == 0.f && c[2] == 0.f && c[3] == 0.f && c[5] == 0.f && c[6] == 0.f && c[7] == 0.f;
    g.Lx = c[0]; g.Ly = c[4]; g.Lz = c[8];
    if (!ortho || !((double)g.Lx > 2 * R) || !((double)g.Ly > 2 * R) || !((double)g.Lz > 2 * R)) {
      post_status(st, FNN_E_CELL, m);
      g.pbc = 0;  // keep the traversal well-defined; the result is flagged invalid
      g.Lx = g.Ly = g.Lz = 0.f;
    }
    ext[0] = g.Lx; ext[1] = g.Ly; ext[2] = g.Lz;
    g.ox = g.oy = g.oz = 0.f;
  }
  if (!g.pbc) {
    if (n == 0) {
      for (int a = 0; a < 6; a++) bb[a] = 0.f;
    }
    g.ox = bb[0]; g.oy = bb[1]; g.oz = bb[2];
    for (int a = 0; a < 3; a++) ext[a] = (double)bb[3 + a] - (double)bb[a];
  }
  // cell counts and spacings in float32 (the edge's 1e-4 margin covers their rounding); the band below
  // stays in float64
  int d[3];
  float fext[3];
  const float fedge = (float)edge;
  for (int a = 0; a < 3; a++) {
    fext[a] = (float)ext[a];
    const float q = fext[a] / fedge;
    d[a] = (q >= 1.f && q < 1e6f) ? (int)floorf(q) : 1;
  }
  long long limit = n > 0 ? 2LL * n : 1;
  while ((long long)d[0] * d[1] * d[2] > limit) {
    int a = (d[0] >= d[1] && d[0] >= d[2]) ? 0 : (d[1] >= d[2] ? 1 : 2);
    d[a] = d[a] * 3 / 4;
    if (d[a] < 1) d[a] = 1;
  }
  g.dx = d[0]; g.dy = d[1]; g.dz = d[2];
  // error band of the float32 predicate, from the largest magnitude S any pair of this structure can
  // present (coordinates, and image offsets |n L| <= 2 max|x| + L/2): twice the bound on the float32
  // error of d2 near R^2, 2 sqrt(3) e R + 3 e^2 + 4 u R^2 with e = 4 u S
  {
    double mabs = 0.0;
    for (int a = 0; a < 3; a++) mabs = fmax(mabs, fmax(fabs((double)bb[a]), fabs((double)bb[3 + a])));
    double Lmax = g.pbc ? fmax(fmax((double)g.Lx, (double)g.Ly), (double)g.Lz) : 0.0;
    double S = g.pbc ? 2.0 * mabs + 0.5 * Lmax + Lmax : mabs;
    const double u = 5.9604644775390625e-8;
    double e = 4.0 * u * S;
    double tau = 2.0 * (3.4641016151377544 * e * R * 1.01 + 3.0 * e * e + 4.0 * u * R * R) + 1e-30;
    g.tau = (float)(tau * (1.0 + 1e-6));
    g.iLx = g.pbc ? 1.f / g.Lx : 0.f;
    g.iLy = g.pbc ? 1.f / g.Ly : 0.f;
    g.iLz = g.pbc ? 1.f / g.Lz : 0.f;
  }
  g.ix = fext[0] > 0.f ? (float)d[0] / fext[0] : 0.f;
  g.iy = fext[1] > 0.f ? (float)d[1] / fext[1] : 0.f;
  g.iz = fext[2] > 0.f ? (float)d[2] / fext[2] : 0.f;
  *cells = d[0] * d[1] * d[2];
  return g;
}

constexpr int SETUP_NT = 512;

__global__ void __launch_bounds__(SETUP_NT) k_mol_setup(fnn_system sys, MolGrid *grid, int32_t *mol_cells,
                                                        int32_t *atom_mol, uint8_t *elem, double R,
                                                        DevStatus *st, const int32_t *bad) {
  const bool drop = *bad != 0;   // inconsistent offsets (posted by k_check_cover): every structure empty
  __shared__ float red[6][SETUP_NT / 32];
  const float4 *pos = reinterpret_cast<const float4 *>(sys.pos);
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int m = blockIdx.x; m < sys.n_mol; m += gridDim.x) {
    int a0 = sys.mol_offsets[m], a1 = sys.mol_offsets[m + 1];
    if (drop || a0 < 0 || a1 < a0 || a1 > sys.n_atoms) {
      if (threadIdx.x == 0) {
        post_status(st, FNN_E_INVALID, m);
        grid[m] = MolGrid{0, 0, 0, 0, 0, 0, 0, 0, 0, 1, 1, 1, 0, 0};
        mol_cells[m] = 1;
      }
      continue;
    }
    int pbc = sys.pbc ? (sys.pbc[m] != 0) : 0;
    float mn[3] = {FLT_MAX, FLT_MAX, FLT_MAX}, mx[3] = {-FLT_MAX, -FLT_MAX, -FLT_MAX};
    for (int i0 = a0 + threadIdx.x; i0 < a1; i0 += 4 * blockDim.x) {
      // four atoms per thread in flight: the loads are issued before any is used
      int zz[4];
      float4 pp[4];
#pragma unroll
      for (int u = 0; u < 4; u++) {
        int i = i0 + u * blockDim.x;
        if (i < a1) {
          zz[u] = sys.Z[i];
          pp[u] = pos[i];
        }
      }
#pragma unroll
      for (int u = 0; u < 4; u++) {
        int i = i0 + u * blockDim.x;
        if (i >= a1) continue;
        atom_mol[i] = m;
        int e = element_of(zz[u]);
        if (e < 0) {
          post_status(st, FNN_E_SPECIES, i);
          e = 0;
        }
        elem[i] = (uint8_t)e;
        float4 p = pp[u];
        if (!isfinite(p.x) || !isfinite(p.y) || !isfinite(p.z)) post_status(st, FNN_E_NONFINITE, i);
        mn[0] = fminf(mn[0], p.x); mn[1] = fminf(mn[1], p.y); mn[2] = fminf(mn[2], p.z);
        mx[0] = fmaxf(mx[0], p.x); mx[1] = fmaxf(mx[1], p.y); mx[2] = fmaxf(mx[2], p.z);
      }
    }
#pragma unroll
    for (int a = 0; a < 3; a++) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        mn[a] = fminf(mn[a], __shfl_xor_sync(FULL, mn[a], o));
        mx[a] = fmaxf(mx[a], __shfl_xor_sync(FULL, mx[a], o));
      }
    }
    if (lane == 0) {
      for (int a = 0; a < 3; a++) { red[a][w] = mn[a]; red[3 + a][w] = mx[a]; }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      for (int k = 1; k < SETUP_NT / 32; k++)
        for (int a = 0; a < 3; a++) {
          red[a][0] = fminf(red[a][0], red[a][k]);
          red[3 + a][0] = fmaxf(red[3 + a][0], red[3 + a][k]);
        }
      float bb[6];
      for (int a = 0; a < 6; a++) bb[a] = red[a][0];
      int cells;
      const MolGrid g = make_grid(sys, m, a1 - a0, pbc, bb, R, st, &cells);
      grid[m] = g;
      mol_cells[m] = cells;
    }
    __syncthreads();
  }
}

__device__ __forceinline__ int axis_cell(float x, float o, float inv, float L, int pbc, int d) {
  float f;
  if (pbc) {
    float xw = x - L * floorf(x / L);
    f = xw * inv;
  } else {
    f = (x - o) * inv;
  }
  f = fminf(fmaxf(f, 0.f), (float)(d - 1));
  return (int)f;
}

__global__ void k_bin(fnn_system sys, const MolGrid *grid, const int32_t *mol_base, const int32_t *atom_mol,
                      int32_t *cell_of, int32_t *cell_count, int64_t cells_bound) {
  const float4 *pos = reinterpret_cast<const float4 *>(sys.pos);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < sys.n_atoms; i += gridDim.x * blockDim.x) {
    int m = atom_mol[i];
    if (m < 0) {  // atom outside every structure: inconsistent offsets (posted by k_check_cover)
      cell_of[i] = -1;
      continue;
    }
    MolGrid g = grid[m];
    float4 p = pos[i];
    int cx = axis_cell(p.x, g.ox, g.ix, g.Lx, g.pbc, g.dx);
    int cy = axis_cell(p.y, g.oy, g.iy, g.Ly, g.pbc, g.dy);
    int cz = axis_cell(p.z, g.oz, g.iz, g.Lz, g.pbc, g.dz);
    int c = mol_base[m] + (cz * g.dy + cy) * g.dx + cx;
    if (c < 0 || c >= cells_bound) {   // unreachable with consistent offsets; never count outside the array
      cell_of[i] = -1;
      continue;
    }
    cell_of[i] = c;
    atomicAdd(&cell_count[c], 1);
  }
}

// cursor[c] starts at cell c's first slot (a copy of the cell starts)
__global__ void k_scatter(int n, const int32_t *cell_of, int32_t *cursor, int32_t *cell_tmp) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    int c = cell_of[i];
    if (c < 0) continue;
    cell_tmp[atomicAdd(&cursor[c], 1)] = i;
  }
}

// one warp per cell: order the cell's atoms by index (rank sort), so traversal order is deterministic;
// their positions are copied in the same order, so the pair search reads candidates contiguously
__global__ void k_sort_cells(const int32_t *meta, const int32_t *cell_start, const int32_t *cell_tmp,
                             const float4 *pos, int32_t *cell_atoms, float4 *cell_pos) {
  int lane = threadIdx.x & 31;
  int ncell = meta[META_CELLS];
  int wg = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
  for (int c = wg; c < ncell; c += nw) {
    int s0 = cell_start[c], s1 = cell_start[c + 1];
    for (int a = s0 + lane; a < s1; a += 32) {
      int v = cell_tmp[a];
      int rank = 0;
      for (int b = s0; b < s1; b++) rank += cell_tmp[b] < v;
      cell_atoms[s0 + rank] = v;
      cell_pos[s0 + rank] = pos[v];
    }
  }
}

// ------------------------------------------------------------------------------------- predicate
struct PredConst {
  double R2d;   // R*R in double (the membership threshold)
  float R2f;    // float(R*R)
  float Rf;
};

// d2 < R^2 with the float64 semantics of the interface, via a float32 test outside a proven band.
// The float32 separation carries an absolute per-component error e <= 4u S (u = 2^-24, S the largest
// magnitude among the coordinates and the image offset); near the threshold the squared distance then
// errs by at most 2 sqrt(3) e R + 3 e^2 + 4 u R^2.  Twice that bound, with S the largest magnitude over
// the whole structure (MolGrid::tau), is the band re-tested in float64.  The image n = -rint(dx / L)
// is formed with 1/L: for a pair within R < L/2, dx/L is far from a half-integer, so n is the same.
// (the image shift n of a pair is returned as floats; make_shift packs it where the pair is kept)
__device__ __forceinline__ bool pair_in(float4 pi, float4 pj, const MolGrid &g, const PredConst &pc, float &nx,
                                        float &ny, float &nz) {
  float dx = pj.x - pi.x, dy = pj.y - pi.y, dz = pj.z - pi.z;
  nx = ny = nz = 0.f;
  if (g.pbc) {
    nx = -rintf(dx * g.iLx);
    ny = -rintf(dy * g.iLy);
    nz = -rintf(dz * g.iLz);
    dx = fmaf(nx, g.Lx, dx);
    dy = fmaf(ny, g.Ly, dy);
    dz = fmaf(nz, g.Lz, dz);
  }
  float d2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
  if (d2 < pc.R2f - g.tau) return true;
  if (d2 > pc.R2f + g.tau) return false;
  // exact float64 predicate, rounded to nearest without contraction
  double rx = __dsub_rn((double)pj.x, (double)pi.x);
  double ry = __dsub_rn((double)pj.y, (double)pi.y);
  double rz = __dsub_rn((double)pj.z, (double)pi.z);
  double ex = __dadd_rn(rx, __dmul_rn((double)nx, (double)g.Lx));
  double ey = __dadd_rn(ry, __dmul_rn((double)ny, (double)g.Ly));
  double ez = __dadd_rn(rz, __dmul_rn((double)nz, (double)g.Lz));
  double D2 = __dadd_rn(__dadd_rn(__dmul_rn(ex, ex), __dmul_rn(ey, ey)), __dmul_rn(ez, ez));
  return D2 < pc.R2d;
}
__device__ __forceinline__ char4 make_shift(float nx, float ny, float nz) {
  return make_char4((signed char)nx, (signed char)ny, (signed char)nz, 0);
}

// entry k of the list stencil() writes, and its length, without the array
__device__ __forceinline__ int stencil_n(int c, int d, int pbc) {
  if (pbc) return d < 3 ? d : 3;
  return 1 + (c > 0) + (c + 1 < d);
}
__device__ __forceinline__ int stencil_at(int c, int d, int pbc, int k) {
  if (pbc) {
    if (d < 3) return k;   // {0} or {0, 1}
    const int v = c - 1 + k;
    return v < 0 ? v + d : (v >= d ? v - d : v);
  }
  return (c > 0 ? c - 1 : c) + k;
}

__device__ __forceinline__ int stencil(int c, int d, int pbc, int *out) {
  if (pbc) {
    if (d == 1) { out[0] = 0; return 1; }
    if (d == 2) { out[0] = 0; out[1] = 1; return 2; }
    out[0] = c == 0 ? d - 1 : c - 1;
    out[1] = c;
    out[2] = c == d - 1 ? 0 : c + 1;
    return 3;
  }
  int n = 0;
  if (c > 0) out[n++] = c - 1;
  out[n++] = c;
  if (c + 1 < d) out[n++] = c + 1;
  return n;
}

// One traversal of atom i's stencil (warp-wide).  Entries are written at base + position while below
// limit; returns the number of neighbours (all of them, written or not).
__device__ __forceinline__ int pairs_row(int i, const float4 *pos, const MolGrid *grid, const int32_t *mol_base,
                                         const int32_t *atom_mol, const int32_t *cell_of,
                                         const int32_t *cell_start, const int32_t *cell_atoms,
                                         const float4 *cell_pos, const PredConst &pc,
                                         int32_t *nbr, char4 *shift, int64_t base, int64_t limit) {
  const int lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1u;
  const int m = atom_mol[i];
  const MolGrid g = grid[m];
  const int mb = mol_base[m];
  const int cl = cell_of[i] - mb;
  const int cx = cl % g.dx, cy = (cl / g.dx) % g.dy, cz = cl / (g.dx * g.dy);
  int ox[3], oy[3], oz[3];
  const int nox = stencil(cx, g.dx, g.pbc, ox), noy = stencil(cy, g.dy, g.pbc, oy), noz = stencil(cz, g.dz, g.pbc, oz);
  const float4 pi = pos[i];
  int count = 0;
  for (int a = 0; a < noz; a++)
    for (int b = 0; b < noy; b++) {
      const int rowc = mb + (oz[a] * g.dy + oy[b]) * g.dx;
      // x-neighbour cells with consecutive indices hold consecutive atoms: one range per run
      for (int q = 0; q < nox;) {
        const int x0 = ox[q];
        int x1 = x0;
        for (q++; q < nox && ox[q] == x1 + 1; q++) x1 = ox[q];
        const int s0 = cell_start[rowc + x0], s1 = cell_start[rowc + x1 + 1];
        for (int k0 = s0; k0 < s1; k0 += 32) {
          const int k = k0 + lane;
          bool in = false;
          int j = -1;
          float nx, ny, nz;
          if (k < s1) {
            const float4 pj = cell_pos[k];
            j = cell_atoms[k];
            in = pair_in(pi, pj, g, pc, nx, ny, nz) && j != i;
          }
          const unsigned mask = __ballot_sync(FULL, in);
          if (in) {
            const int64_t idx = base + count + __popc(mask & lt);
            if (idx < limit) {
              nbr[idx] = j;
              shift[idx] = make_shift(nx, ny, nz);
            }
          }
          count += __popc(mask);
        }
      }
    }
  return count;
}

// Two-traversal form (the allocation-free entry point): COUNT writes each atom's count, FILL writes the
// entries at the CSR row pointers.
template <bool FILL>
__global__ void __launch_bounds__(256) k_pairs(fnn_system sys, const MolGrid *grid, const int32_t *mol_base,
                                               const int32_t *atom_mol, const int32_t *cell_of,
                                               const int32_t *cell_start, const int32_t *cell_atoms,
                                               const float4 *cell_pos, PredConst pc, int32_t *counts,
                                               const int32_t *row_ptr,
                                               int32_t *nbr, char4 *shift, int64_t cap, const int32_t *meta) {
  const float4 *pos = reinterpret_cast<const float4 *>(sys.pos);
  const int lane = threadIdx.x & 31;
  const int wg = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
  const int n_binned = cell_start[meta[META_CELLS]];   // atoms that belong to a structure
  for (int w = wg; w < n_binned; w += nw) {
    const int i = cell_atoms[w];   // atoms in cell order: neighbouring warps share neighbour cells
    const int64_t out = FILL ? (int64_t)row_ptr[i] : 0;
    const int count = pairs_row(i, pos, grid, mol_base, atom_mol, cell_of, cell_start, cell_atoms, cell_pos, pc, nbr, shift,
                                out, FILL ? cap : 0);
    if (!FILL && lane == 0) counts[i] = count;
  }
}

// PAIR_STRIDE (fnn_internal.cuh): staged entries per atom; longer rows are traversed again at compaction

// pass 1, a block per cell (or per slice of a cell's centres when there are fewer cells than blocks): the
// cell's stencil candidates (positions and atoms, in the traversal order of
// pairs_row) are staged in shared memory once and tested by each warp against its centre atoms of the
// cell, so every centre's row comes out exactly as pairs_row writes it: into the atom's own
// PAIR_STRIDE-entry slot of the staging buffer, with its count.  A cell whose stencil holds more than
// CELL_CAND candidates is traversed per centre from global memory instead.
constexpr int CELL_WARPS = 4, CELL_CAND = 1024;

__global__ void __launch_bounds__(CELL_WARPS * 32, 8) k_pairs_stage(fnn_system sys, const MolGrid *grid,
                                                                 const int32_t *mol_base, const int32_t *atom_mol,
                                                                 const int32_t *cell_of, const int32_t *cell_start,
                                                                 const int32_t *cell_atoms, const float4 *cell_pos,
                                                                 PredConst pc, int32_t *counts, int32_t *tnbr,
                                                                 char4 *tshift, const int32_t *meta) {
  __shared__ float4 cpos[CELL_CAND];
  __shared__ int32_t cidx[CELL_CAND];
  __shared__ int32_t run_s0[27], run_off[28], run_total;   // at most 9 stencil rows of at most 3 runs
  const float4 *pos = reinterpret_cast<const float4 *>(sys.pos);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const unsigned lt = (1u << lane) - 1u;
  const int n_cells = meta[META_CELLS];
  // with fewer cells than blocks, S blocks share a cell, block slice sl taking its centres sl, sl + S, ...
  const int S = n_cells > 0 ? max(1, min(8, (int)gridDim.x / n_cells)) : 1;
  for (int t = blockIdx.x; t < n_cells * S; t += gridDim.x) {
    const int c = t / S, sl = t - c * S;
    const int a0 = cell_start[c], a1 = cell_start[c + 1];
    if (a0 + sl * CELL_WARPS >= a1) continue;   // no centres for this slice (uniform over the block)
    const int m = atom_mol[cell_atoms[a0]];
    const MolGrid g = grid[m];
    const int mb = mol_base[m];
    const int cl = c - mb;
    const int cx = cl % g.dx, cy = (cl / g.dx) % g.dy, cz = cl / (g.dx * g.dy);
    const int noy = stencil_n(cy, g.dy, g.pbc), noz = stencil_n(cz, g.dz, g.pbc);
    // x-neighbour cells with consecutive indices hold consecutive atoms: the (at most three) runs of the
    // x stencil, grouped as pairs_row groups them
    const int nox = stencil_n(cx, g.dx, g.pbc);
    const int x0 = stencil_at(cx, g.dx, g.pbc, 0), x1 = stencil_at(cx, g.dx, g.pbc, 1),
              x2 = stencil_at(cx, g.dx, g.pbc, 2);
    int ra0 = x0, ra1 = x0, rb0 = 0, rb1 = -1, rc0 = 0, rc1 = -1, nxr = 1;
    if (nox > 1) {
      if (x1 == ra1 + 1) ra1 = x1;
      else { rb0 = rb1 = x1; nxr = 2; }
    }
    if (nox > 2) {
      if (nxr == 1) {
        if (x2 == ra1 + 1) ra1 = x2;
        else { rb0 = rb1 = x2; nxr = 2; }
      } else {
        if (x2 == rb1 + 1) rb1 = x2;
        else { rc0 = rc1 = x2; nxr = 3; }
      }
    }
    __syncthreads();   // the previous cell's candidates and run table are no longer read
    if (warp == 0) {
      // lane t: stencil row t (z-major, as pairs_row walks it), its runs' ranges loaded side by side;
      // the table holds each run's first candidate and its offset in the traversal order
      const int nrow = noz * noy;
      int s0 = 0, s1 = 0, s2 = 0, l0 = 0, l1 = 0, l2 = 0;
      if (lane < nrow) {
        const int a = lane / noy, b = lane - a * noy;
        const int rowc = mb + (stencil_at(cz, g.dz, g.pbc, a) * g.dy + stencil_at(cy, g.dy, g.pbc, b)) * g.dx;
        s0 = cell_start[rowc + ra0];
        l0 = cell_start[rowc + ra1 + 1] - s0;
        if (nxr > 1) {
          s1 = cell_start[rowc + rb0];
          l1 = cell_start[rowc + rb1 + 1] - s1;
        }
        if (nxr > 2) {
          s2 = cell_start[rowc + rc0];
          l2 = cell_start[rowc + rc1 + 1] - s2;
        }
      }
      const int mine = l0 + l1 + l2;
      int inc = mine;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(FULL, inc, o);
        if (lane >= o) inc += v;
      }
      const int ex = inc - mine;
      if (lane < nrow) {
        const int r = lane * nxr;
        run_s0[r] = s0;
        run_off[r] = ex;
        if (nxr > 1) {
          run_s0[r + 1] = s1;
          run_off[r + 1] = ex + l0;
        }
        if (nxr > 2) {
          run_s0[r + 2] = s2;
          run_off[r + 2] = ex + l0 + l1;
        }
      }
      if (lane == 31) {
        run_off[nrow * nxr] = inc;
        run_total = inc;
      }
    }
    __syncthreads();
    const int total = run_total;
    if (total <= CELL_CAND) {
      // candidates in traversal order: each thread finds the run of its slots in the table (its slots
      // ascend, so the search only moves forward) and has two loads in flight before it stores
      int r = 0;
      for (int h = 0; h < total; h += 2 * CELL_WARPS * 32) {
        float4 v[2];
        int id[2];
#pragma unroll
        for (int u = 0; u < 2; u++) {
          const int k = h + threadIdx.x + u * CELL_WARPS * 32;
          if (k < total) {
            while (run_off[r + 1] <= k) r++;
            const int src = run_s0[r] + (k - run_off[r]);
            v[u] = cell_pos[src];
            id[u] = cell_atoms[src];
          }
        }
#pragma unroll
        for (int u = 0; u < 2; u++) {
          const int k = h + threadIdx.x + u * CELL_WARPS * 32;
          if (k < total) {
            cpos[k] = v[u];
            cidx[k] = id[u];
          }
        }
      }
      __syncthreads();
      for (int w = a0 + sl * CELL_WARPS + warp; w < a1; w += S * CELL_WARPS) {
        const int i = cell_atoms[w];
        const float4 pi = cell_pos[w];   // pos[i], copied in cell order: no wait on i
        const int64_t base = (int64_t)i * PAIR_STRIDE;
        int count = 0;
        for (int k0 = 0; k0 < total; k0 += 32) {
          const int k = k0 + lane;
          bool in = false;
          int j = -1;
          float nx, ny, nz;
          if (k < total) {
            j = cidx[k];
            in = pair_in(pi, cpos[k], g, pc, nx, ny, nz) && j != i;
          }
          const unsigned mask = __ballot_sync(FULL, in);
          if (in) {
            const int at = count + __popc(mask & lt);
            if (at < PAIR_STRIDE) {
              tnbr[base + at] = j;
              tshift[base + at] = make_shift(nx, ny, nz);
            }
          }
          count += __popc(mask);
        }
        if (lane == 0) counts[i] = count;
      }
    } else {
      for (int w = a0 + sl * CELL_WARPS + warp; w < a1; w += S * CELL_WARPS) {
        const int i = cell_atoms[w];
        const int64_t base = (int64_t)i * PAIR_STRIDE;
        const int count = pairs_row(i, pos, grid, mol_base, atom_mol, cell_of, cell_start, cell_atoms, cell_pos, pc,
                                    tnbr, tshift, base, base + PAIR_STRIDE);
        if (lane == 0) counts[i] = count;
      }
    }
  }
}

// pass 2: staged rows copied to their CSR place (row_ptr from the scan of the counts), sorted by
// neighbour element (a stable counting sort: ballots count, then place, each element's entries); a row
// longer than the slot is found again by a second traversal writing straight into the list
__global__ void __launch_bounds__(256) k_pairs_compact(fnn_system sys, const MolGrid *grid, const int32_t *mol_base,
                                                       const int32_t *atom_mol, const int32_t *cell_of,
                                                       const int32_t *cell_start, const int32_t *cell_atoms,
                                                       const float4 *cell_pos, PredConst pc, const int32_t *row_ptr,
                                                       const int32_t *tnbr,
                                                       const char4 *tshift, const uint8_t *elem, int32_t *nbr,
                                                       char4 *shift, int64_t cap, const int32_t *meta) {
  const float4 *pos = reinterpret_cast<const float4 *>(sys.pos);
  const int lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1u;
  const int wg = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
  const int n_binned = cell_start[meta[META_CELLS]];
  for (int w = wg; w < n_binned; w += nw) {
    const int i = cell_atoms[w];
    const int64_t dst = row_ptr[i];
    const int n = row_ptr[i + 1] - row_ptr[i];
    if (n <= PAIR_STRIDE) {
      // the whole staged row in registers (all its loads in flight together), then a stable counting
      // sort by neighbour element: ballots count each element's entries, then place them
      constexpr int NCH = PAIR_STRIDE / 32;
      const int64_t src = (int64_t)i * PAIR_STRIDE;
      int jv[NCH], ev[NCH];
      char4 sv[NCH];
#pragma unroll
      for (int c = 0; c < NCH; c++) {
        const int k = 32 * c + lane;
        jv[c] = 0;
        sv[c] = make_char4(0, 0, 0, 0);
        if (k < n) {
          jv[c] = tnbr[src + k];
          sv[c] = tshift[src + k];
        }
      }
#pragma unroll
      for (int c = 0; c < NCH; c++) ev[c] = 32 * c + lane < n ? (int)elem[jv[c]] : 0;
      // the counts one element per lane, from three ballots of the entries' element bits
      int cnt = 0;
#pragma unroll
      for (int c = 0; c < NCH; c++) {
        if (32 * c >= n) break;   // uniform over the warp
        const unsigned vm = __ballot_sync(FULL, 32 * c + lane < n);
        cnt += __popc(elem_lanes(lane, __ballot_sync(FULL, ev[c] & 1), __ballot_sync(FULL, ev[c] & 2),
                                 __ballot_sync(FULL, ev[c] & 4)) & vm);
      }
      if (lane >= NE) cnt = 0;
      int run = cnt;   // exclusive scan over lanes 0 .. NE - 1: lane q's next place for element q
#pragma unroll
      for (int o = 1; o < 8; o <<= 1) {
        const int v = __shfl_up_sync(FULL, run, o);
        if (lane >= o) run += v;
      }
      run -= cnt;
#pragma unroll
      for (int c = 0; c < NCH; c++) {
        if (32 * c >= n) break;
        const unsigned vm = __ballot_sync(FULL, 32 * c + lane < n);
        const unsigned b0 = __ballot_sync(FULL, ev[c] & 1), b1 = __ballot_sync(FULL, ev[c] & 2),
                       b2 = __ballot_sync(FULL, ev[c] & 4);
        const int at = __shfl_sync(FULL, run, ev[c]) + __popc(elem_lanes(ev[c], b0, b1, b2) & vm & lt);
        run += __popc(elem_lanes(lane, b0, b1, b2) & vm);
        if (32 * c + lane < n && dst + at < cap) {
          nbr[dst + at] = jv[c];
          shift[dst + at] = sv[c];
        }
      }
    } else {
      pairs_row(i, pos, grid, mol_base, atom_mol, cell_of, cell_start, cell_atoms, cell_pos, pc, nbr, shift, dst, cap);
    }
  }
}

// ------------------------------------------------------------------ small systems: the build in one block
// At most SMALL_BUILD_ATOMS atoms in SMALL_BUILD_MOL structures: every stage of the build in one block of
// 1024 threads -- the global offsets check, per-atom setup, per-structure images and predicate band
// (make_grid), each atom's neighbours by brute force over its structure with the same predicate
// (pair_in: the same set), row offsets by a block scan, rows of at most PAIR_STRIDE entries sorted by
// neighbour element (stable; longer rows in atom order), and the species order of the networks.
// One launch instead of the cell-list pipeline's thirteen, for systems whose cost is launch latency.
constexpr int SMALL_NT = 1024;
struct SmallBuildShared {
  float4 pos[SMALL_BUILD_ATOMS];
  int32_t z[SMALL_BUILD_ATOMS];
  int32_t off[SMALL_BUILD_MOL + 1];
  float bb[SMALL_BUILD_MOL][6];
  MolGrid g[SMALL_BUILD_MOL];
  int32_t am[SMALL_BUILD_ATOMS];
  int32_t start[SMALL_BUILD_ATOMS + 1];
  uint8_t el[SMALL_BUILD_ATOMS];
  int32_t stage_j[SMALL_NT / 32][PAIR_STRIDE];
  char4 stage_s[SMALL_NT / 32][PAIR_STRIDE];
  int ecount[8], eseg[8];
  int wcnt[SMALL_NT / 32][8];
};
static_assert(SMALL_BUILD_ATOMS <= SMALL_NT, "one atom per thread in the scans");

__global__ void __launch_bounds__(SMALL_NT, 1)
    k_small_build(fnn_system sys, double R, PredConst pc, int64_t cap, int32_t *atom_mol, uint8_t *elem,
                  MolGrid *grid, int32_t *row_ptr, int32_t *nbr, char4 *shift, int32_t *perm, int32_t *inv,
                  int32_t *tile_elem, int ntiles_cap, int pad_cap, int32_t *meta, DevStatus *st) {
  extern __shared__ __align__(16) unsigned char small_build_dyn[];
  SmallBuildShared &S = *reinterpret_cast<SmallBuildShared *>(small_build_dyn);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarp = SMALL_NT / 32;
  const unsigned lt = (1u << lane) - 1u;
  const int N = sys.n_atoms, NM = sys.n_mol;
  // positions, atomic numbers and offsets read once into shared memory
  const float4 *gpos = reinterpret_cast<const float4 *>(sys.pos);
  for (int i = tid; i < N; i += SMALL_NT) {
    S.pos[i] = gpos[i];
    S.z[i] = sys.Z[i];
  }
  for (int m = tid; m <= NM; m += SMALL_NT) S.off[m] = sys.mol_offsets[m];
  __syncthreads();
  const float4 *pos = S.pos;
  const int32_t *offs = S.off;
  // offsets start at 0, end at N and never decrease; otherwise no atom belongs to a structure
  int badl = 0;
  for (int m = tid; m <= NM; m += SMALL_NT) {
    const int a = offs[m];
    bool ok = (m == 0) ? a == 0 : (a >= offs[m - 1]);
    if (m == NM) ok = ok && a == N;
    if (!ok) {
      post_status(st, FNN_E_INVALID, m);
      badl = 1;
    }
  }
  for (int m = tid; m < NM; m += SMALL_NT)
    for (int a = 0; a < 3; a++) {
      S.bb[m][a] = __int_as_float(0x7f800000);
      S.bb[m][3 + a] = __int_as_float((int)0xff800000);
    }
  if (tid < 8) S.ecount[tid] = 0;
  const bool bad = __syncthreads_or(badl) != 0;
  // per atom: structure, element, checks, bounding boxes
  for (int i = tid; i < N; i += SMALL_NT) {
    int m = -1, e = 0;
    if (!bad) {
      int lo = 0, hi = NM;
      while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (offs[mid] <= i) lo = mid; else hi = mid;
      }
      if (offs[lo] <= i && i < offs[lo + 1]) m = lo;
    }
    if (m >= 0) {
      e = element_of(S.z[i]);
      if (e < 0) {
        post_status(st, FNN_E_SPECIES, i);
        e = 0;
      }
      const float4 p = pos[i];
      if (!isfinite(p.x) || !isfinite(p.y) || !isfinite(p.z)) post_status(st, FNN_E_NONFINITE, i);
      atomic_fmin(&S.bb[m][0], p.x);
      atomic_fmin(&S.bb[m][1], p.y);
      atomic_fmin(&S.bb[m][2], p.z);
      atomic_fmax(&S.bb[m][3], p.x);
      atomic_fmax(&S.bb[m][4], p.y);
      atomic_fmax(&S.bb[m][5], p.z);
    }
    S.am[i] = m;
    S.el[i] = (uint8_t)e;
    atom_mol[i] = m;
    elem[i] = (uint8_t)e;
    atomicAdd(&S.ecount[e], 1);
  }
  __syncthreads();
  // per structure: images and the predicate band, exactly as the cell-list build takes them
  for (int m = tid; m < NM; m += SMALL_NT) {
    const int a0 = offs[m], a1 = offs[m + 1];
    MolGrid g = MolGrid{0, 0, 0, 0, 0, 0, 0, 0, 0, 1, 1, 1, 0, 0};
    if (!bad && a0 >= 0 && a1 >= a0 && a1 <= N) {
      const int pbc = sys.pbc ? (sys.pbc[m] != 0) : 0;
      float bb[6];
      for (int a = 0; a < 6; a++) bb[a] = S.bb[m][a];
      int cells;
      g = make_grid(sys, m, a1 - a0, pbc, bb, R, st, &cells);
    }
    S.g[m] = g;
    grid[m] = g;
  }
  __syncthreads();
  // pass 1: neighbour counts, a warp per atom over the atoms of its structure
  for (int i = warp; i < N; i += nwarp) {
    const int m = S.am[i];
    int count = 0;
    if (m >= 0) {
      const MolGrid g = S.g[m];
      const float4 pi = pos[i];
      const int a0 = offs[m], a1 = offs[m + 1];
      for (int j0 = a0; j0 < a1; j0 += 32) {
        const int j = j0 + lane;
        bool in = false;
        float nx, ny, nz;
        if (j < a1) in = pair_in(pi, pos[j], g, pc, nx, ny, nz) && j != i;
        count += __popc(__ballot_sync(FULL, in));
      }
    }
    if (lane == 0) S.start[i] = count;
  }
  __syncthreads();
  // row offsets and the entry count
  {
    const int v = tid < N ? S.start[tid] : 0;
    int tot;
    const int ex = block_excl_scan<SMALL_NT>(v, &tot);
    if (tid < N) {
      S.start[tid] = ex;
      row_ptr[tid] = ex;
    }
    if (tid == 0) {
      S.start[N] = tot;
      row_ptr[N] = tot;
      meta[META_NNZ] = tot;
      if ((int64_t)tot > cap) post_status(st, FNN_E_CAPACITY, tot);
    }
  }
  __syncthreads();
  // pass 2: the entries (none when the list is over capacity: the status says so)
  const bool fill = (int64_t)S.start[N] <= cap;
  for (int i = warp; fill && i < N; i += nwarp) {
    const int m = S.am[i];
    if (m < 0) continue;   // uniform over the warp
    const MolGrid g = S.g[m];
    const float4 pi = pos[i];
    const int a0 = offs[m], a1 = offs[m + 1];
    const int64_t dst = S.start[i];
    const int n = S.start[i + 1] - S.start[i];
    const bool sortable = n <= PAIR_STRIDE;
    int at = 0;
    for (int j0 = a0; j0 < a1; j0 += 32) {
      const int j = j0 + lane;
      bool in = false;
      float nx = 0.f, ny = 0.f, nz = 0.f;
      if (j < a1) in = pair_in(pi, pos[j], g, pc, nx, ny, nz) && j != i;
      const unsigned mask = __ballot_sync(FULL, in);
      if (in) {
        const int idx = at + __popc(mask & lt);
        if (sortable) {
          S.stage_j[warp][idx] = j;
          S.stage_s[warp][idx] = make_shift(nx, ny, nz);
        } else {
          nbr[dst + idx] = j;
          shift[dst + idx] = make_shift(nx, ny, nz);
        }
      }
      at += __popc(mask);
    }
    __syncwarp();
    if (sortable) {   // stable counting sort of the staged row by neighbour element
      // (the counts one element per lane, from three ballots of the entries' element bits)
      constexpr int NCH = PAIR_STRIDE / 32;
      int jv[NCH], ev[NCH];
      char4 sv[NCH];
      int cnt = 0;   // lane q < NE: entries of element q
#pragma unroll
      for (int c = 0; c < NCH; c++) {
        if (32 * c >= n) break;   // uniform over the warp
        const int k = 32 * c + lane;
        jv[c] = k < n ? S.stage_j[warp][k] : 0;
        sv[c] = k < n ? S.stage_s[warp][k] : make_char4(0, 0, 0, 0);
        ev[c] = k < n ? (int)S.el[jv[c]] : 0;
        const unsigned vm = __ballot_sync(FULL, k < n);
        cnt += __popc(elem_lanes(lane, __ballot_sync(FULL, ev[c] & 1), __ballot_sync(FULL, ev[c] & 2),
                                 __ballot_sync(FULL, ev[c] & 4)) & vm);
      }
      if (lane >= NE) cnt = 0;
      int run = cnt;   // exclusive scan over lanes 0 .. NE - 1: lane q's next place for element q
#pragma unroll
      for (int o = 1; o < 8; o <<= 1) {
        const int v = __shfl_up_sync(FULL, run, o);
        if (lane >= o) run += v;
      }
      run -= cnt;
#pragma unroll
      for (int c = 0; c < NCH; c++) {
        if (32 * c >= n) break;
        const int k = 32 * c + lane;
        const unsigned vm = __ballot_sync(FULL, k < n);
        const unsigned b0 = __ballot_sync(FULL, ev[c] & 1), b1 = __ballot_sync(FULL, ev[c] & 2),
                       b2 = __ballot_sync(FULL, ev[c] & 4);
        const int w = __shfl_sync(FULL, run, ev[c]) + __popc(elem_lanes(ev[c], b0, b1, b2) & vm & lt);
        run += __popc(elem_lanes(lane, b0, b1, b2) & vm);
        if (k < n) {
          nbr[dst + w] = jv[c];
          shift[dst + w] = sv[c];
        }
      }
    }
    __syncwarp();
  }
  // species order: element segments padded to ROW_TILE rows, atoms in index order within each
  if (tid == 0) {
    int s0 = 0;
    for (int e = 0; e < NE; e++) {
      S.eseg[e] = s0;
      meta[META_SEG + e] = s0;
      s0 += (S.ecount[e] + ROW_TILE - 1) / ROW_TILE * ROW_TILE;
    }
    S.eseg[NE] = s0;
    meta[META_SEG + NE] = s0;
    meta[META_NPAD] = s0;
  }
  for (int r = tid; r < pad_cap; r += SMALL_NT) inv[r] = -1;
  __syncthreads();
  {   // rank among the atoms of the same element, in index order: ballots per warp, then the warps before
    const int e_i = tid < N ? (int)S.el[tid] : NE;
    int mine = 0;
    for (int q = 0; q < NE; q++) {
      const unsigned mq = __ballot_sync(FULL, e_i == q);
      if (lane == 0) S.wcnt[warp][q] = __popc(mq);
      if (e_i == q) mine = __popc(mq & lt);
    }
    __syncthreads();
    if (tid < N) {
      int before = 0;
      for (int w = 0; w < warp; w++) before += S.wcnt[w][e_i];
      const int row = S.eseg[e_i] + before + mine;
      perm[tid] = row;
      inv[row] = tid;
    }
  }
  for (int t = tid; t < ntiles_cap; t += SMALL_NT) {
    const int r = t * ROW_TILE;
    int e = -1;
    for (int q = 0; q < NE; q++)
      if (r >= S.eseg[q] && r < S.eseg[q + 1]) e = q;
    tile_elem[t] = e;
  }
}

// rows of at most PAIR_STRIDE entries sorted by neighbour element in place (stable), as the staged
// compaction leaves them: the whole row is read into registers before any entry is written back
__global__ void __launch_bounds__(256) k_sort_rows(int n_atoms, const int32_t *row_ptr, const uint8_t *elem,
                                                   int32_t *nbr, char4 *shift, int64_t cap) {
  constexpr int NCH = PAIR_STRIDE / 32;
  const int lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1u;
  const int wg = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
  for (int i = wg; i < n_atoms; i += nw) {
    const int64_t b0 = row_ptr[i];
    const int n = row_ptr[i + 1] - row_ptr[i];
    if (n > PAIR_STRIDE || b0 + n > cap) continue;   // long rows stay in traversal order
    int jv[NCH], ev[NCH];
    char4 sv[NCH];
    int off[NE];
#pragma unroll
    for (int q = 0; q < NE; q++) off[q] = 0;
#pragma unroll
    for (int c = 0; c < NCH; c++) {
      const int k = 32 * c + lane;
      jv[c] = 0;
      ev[c] = -1;
      sv[c] = make_char4(0, 0, 0, 0);
      if (k < n) {
        jv[c] = nbr[b0 + k];
        sv[c] = shift[b0 + k];
        ev[c] = elem[jv[c]];
      }
#pragma unroll
      for (int q = 0; q < NE; q++) off[q] += __popc(__ballot_sync(FULL, ev[c] == q));
    }
    int run = 0;
#pragma unroll
    for (int q = 0; q < NE; q++) {
      const int cq = off[q];
      off[q] = run;
      run += cq;
    }
    __syncwarp();
#pragma unroll
    for (int c = 0; c < NCH; c++) {
      int at = 0;
#pragma unroll
      for (int q = 0; q < NE; q++) {
        const unsigned mq = __ballot_sync(FULL, ev[c] == q);
        if (ev[c] == q) at = off[q] + __popc(mq & lt);
        off[q] += __popc(mq);
      }
      if (ev[c] >= 0) {
        nbr[b0 + at] = jv[c];
        shift[b0 + at] = sv[c];
      }
    }
  }
}

__global__ void k_check_capacity(const int32_t *row_ptr, int n, int64_t cap, int32_t *meta, DevStatus *st) {
  int64_t nnz = row_ptr[n];
  meta[META_NNZ] = (int32_t)nnz;
  if (nnz > cap) post_status(st, FNN_E_CAPACITY, nnz);
}

// ---------------------------------------------------------------------------- species segments
constexpr int ELEM_NT = 256;

__global__ void k_elem_count(int n, const uint8_t *elem, int32_t *blk_count) {
  __shared__ int c[8];
  if (threadIdx.x < 8) c[threadIdx.x] = 0;
  __syncthreads();
  int i = blockIdx.x * ELEM_NT + threadIdx.x;
  if (i < n) atomicAdd(&c[elem[i]], 1);
  __syncthreads();
  if (threadIdx.x < 8) blk_count[blockIdx.x * 8 + threadIdx.x] = c[threadIdx.x];
}

// single block: per-element exclusive scan over blocks, padded segment starts, tile table
__global__ void k_elem_scan(int nblk, int32_t *blk_count, int32_t *meta, int32_t *tile_elem, int ntiles_cap) {
  __shared__ int totals[8];
  for (int e = 0; e < NE; e++) {
    int carry = 0;
    for (int c = 0; c < nblk; c += SCAN_NT) {
      int k = c + threadIdx.x;
      int v = k < nblk ? blk_count[k * 8 + e] : 0;
      int tot;
      int ex = block_excl_scan<SCAN_NT>(v, &tot);
      if (k < nblk) blk_count[k * 8 + e] = ex + carry;
      carry += tot;
    }
    if (threadIdx.x == 0) totals[e] = carry;
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    int s = 0;
    for (int e = 0; e < NE; e++) {
      meta[META_SEG + e] = s;
      s += (totals[e] + ROW_TILE - 1) / ROW_TILE * ROW_TILE;
    }
    meta[META_SEG + NE] = s;
    meta[META_NPAD] = s;
  }
  __syncthreads();
  for (int t = threadIdx.x; t < ntiles_cap; t += blockDim.x) {
    int r = t * ROW_TILE, e = -1;
    for (int q = 0; q < NE; q++)
      if (r >= meta[META_SEG + q] && r < meta[META_SEG + q + 1]) e = q;
    tile_elem[t] = e;
  }
}

__global__ void k_elem_scatter(int n, const uint8_t *elem, const int32_t *blk_off, const int32_t *meta,
                               int32_t *perm, int32_t *inv) {
  __shared__ int wcnt[ELEM_NT / 32][8];
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int i = blockIdx.x * ELEM_NT + threadIdx.x;
  int e = i < n ? elem[i] : 7;
  unsigned lt = (1u << lane) - 1u;
  int my_rank = 0;
  for (int q = 0; q < NE; q++) {
    unsigned mask = __ballot_sync(FULL, e == q);
    if (lane == 0) wcnt[w][q] = __popc(mask);
    if (e == q) my_rank = __popc(mask & lt);
  }
  __syncthreads();
  if (i < n) {
    int before = 0;
    for (int k = 0; k < w; k++) before += wcnt[k][e];
    int row = meta[META_SEG + e] + blk_off[blockIdx.x * 8 + e] + before + my_rank;
    perm[i] = row;
    inv[row] = i;
  }
}

// ------------------------------------------------------------------------------------------ host
template <typename T>
static fnn_status grow(fnn_ctx *ctx, T **p, size_t count) {
  if (*p) cudaFree(*p);
  *p = nullptr;
  if (count == 0) count = 1;
  if (cudaMalloc((void **)p, count * sizeof(T)) != cudaSuccess) {
    cudaGetLastError();
    ctx->last_error = "cudaMalloc failed for neighbour-list storage";
    return FNN_E_OOM;
  }
  return FNN_OK;
}

static fnn_status reserve(fnn_nlist *nl, int32_t n_atoms, int32_t n_mol, int64_t capacity) {
  fnn_ctx *ctx = nl->ctx;
  fnn_status st;
  if (n_atoms > nl->atom_cap || !nl->perm) {
    int32_t na = n_atoms > nl->atom_cap ? n_atoms : nl->atom_cap;
    if ((st = grow(ctx, &nl->row_ptr, (size_t)na + 1)) || (st = grow(ctx, &nl->atom_mol, na)) ||
        (st = grow(ctx, &nl->elem, na)) || (st = grow(ctx, &nl->cell_of, na)) ||
        (st = grow(ctx, &nl->cell_tmp, na)) || (st = grow(ctx, &nl->cell_atoms, na)) ||
        (st = grow(ctx, &nl->cell_pos, na)) ||
        (st = grow(ctx, &nl->counts, (size_t)na + 1)) || (st = grow(ctx, &nl->perm, na)))
      return st;
    int32_t pad = (na + ROW_TILE - 1) / ROW_TILE * ROW_TILE + NE * ROW_TILE;
    int32_t nblk = (na + ELEM_NT - 1) / ELEM_NT + 1;
    if ((st = grow(ctx, &nl->inv, pad)) || (st = grow(ctx, &nl->tile_elem, pad / ROW_TILE)) ||
        (st = grow(ctx, &nl->blk_count, (size_t)nblk * 8)))
      return st;
    if ((st = grow(ctx, &nl->stage_nbr, (size_t)na * PAIR_STRIDE)) ||
        (st = grow(ctx, &nl->stage_shift, (size_t)na * PAIR_STRIDE)))
      return st;
    nl->atom_cap = na;
    nl->pad_cap = pad;
  }
  if (n_mol > nl->mol_cap || !nl->grid) {
    int32_t nm = n_mol > nl->mol_cap ? n_mol : nl->mol_cap;
    if ((st = grow(ctx, &nl->grid, nm)) || (st = grow(ctx, &nl->mol_cells, (size_t)nm + 1)) ||
        (st = grow(ctx, &nl->bbox, (size_t)6 * nm)))
      return st;
    nl->mol_cap = nm;
  }
  int32_t cells = 2 * nl->atom_cap + nl->mol_cap + 1;
  if (cells > nl->cell_cap) {
    if ((st = grow(ctx, &nl->cell_count, (size_t)cells + 1)) || (st = grow(ctx, &nl->cell_start, (size_t)cells + 1)))
      return st;
    nl->cell_cap = cells;
  }
  int64_t need_tmp = scan_tmp_needed((int64_t)cells + 1);
  int64_t t2 = scan_tmp_needed((int64_t)nl->atom_cap + 1);
  int64_t t3 = scan_tmp_needed((int64_t)nl->mol_cap + 1);
  if (t2 > need_tmp) need_tmp = t2;
  if (t3 > need_tmp) need_tmp = t3;
  need_tmp *= 3;   // one region each for the structure, cell and row scans of a build
  if (need_tmp > nl->scan_tmp_len) {
    if ((st = grow(ctx, &nl->scan_tmp, need_tmp))) return st;
    nl->scan_tmp_len = need_tmp;
  }
  if (!nl->meta) {
    if ((st = grow(ctx, &nl->meta, META_LEN))) return st;
    cudaMemset(nl->meta, 0, META_LEN * sizeof(int32_t));
  }
  if (capacity > nl->capacity) {
    if ((st = grow(ctx, &nl->nbr, capacity)) || (st = grow(ctx, &nl->shift, capacity))) return st;
    nl->capacity = capacity;
  }
  return FNN_OK;
}

}  // namespace fnn

using namespace fnn;

extern "C" fnn_status fnn_nlist_create(fnn_ctx *ctx, fnn_nlist **out, int64_t capacity) {
  if (!ctx || !out || capacity < 0) return FNN_E_INVALID;
  fnn_nlist *nl = new fnn_nlist();
  nl->ctx = ctx;
  nl->auto_size = capacity == 0;
  if (capacity > 0) {
    fnn_status st = reserve(nl, 0, 0, capacity);
    if (st) {
      fnn_nlist_destroy(nl);
      return st;
    }
  }
  *out = nl;
  return FNN_OK;
}

extern "C" fnn_status fnn_nlist_destroy(fnn_nlist *nl) {
  if (!nl) return FNN_E_INVALID;
  void *ptrs[] = {nl->row_ptr, nl->nbr, nl->shift, nl->atom_mol, nl->elem, nl->cell_of, nl->cell_tmp,
                  nl->cell_atoms, nl->counts, nl->grid, nl->mol_cells, nl->cell_count, nl->cell_start,
                  nl->perm, nl->inv, nl->tile_elem, nl->blk_count, nl->meta, nl->scan_tmp, nl->stage_nbr,
                  nl->stage_shift, nl->bbox, nl->cell_pos};
  for (void *p : ptrs)
    if (p) cudaFree(p);
  delete nl;
  return FNN_OK;
}

extern "C" fnn_status fnn_nlist_reserve(fnn_nlist *nl, int32_t n_atoms, int32_t n_mol, int64_t capacity) {
  if (!nl || n_atoms < 0 || n_mol < 0 || capacity < 0) return FNN_E_INVALID;
  return reserve(nl, n_atoms, n_mol, capacity);
}

static fnn_status validate_system(fnn_ctx *ctx, const fnn_system *sys) {
  if (!sys || sys->n_atoms < 0 || sys->n_mol < 1 || !sys->mol_offsets) {
    ctx->last_error = "invalid system descriptor";
    return FNN_E_INVALID;
  }
  if (sys->n_atoms > 0 && (!sys->Z || !sys->pos)) {
    ctx->last_error = "system without species or positions";
    return FNN_E_INVALID;
  }
  if (((uintptr_t)sys->pos & 15) != 0) {
    ctx->last_error = "positions must be 16-byte aligned float4";
    return FNN_E_INVALID;
  }
  if (sys->pbc && !sys->cell) {
    ctx->last_error = "pbc flags without cells";
    return FNN_E_INVALID;
  }
  return FNN_OK;
}

extern "C" fnn_status fnn_build_neighbors(fnn_ctx *ctx, const fnn_system *sys, fnn_nlist *nl, void *stream) {
  if (!ctx || !nl || nl->ctx != ctx) return FNN_E_INVALID;
  fnn_status st = validate_system(ctx, sys);
  if (st) return st;
  cudaStream_t s = (cudaStream_t)stream;
  const int N = sys->n_atoms, NM = sys->n_mol;
  int64_t cap = nl->capacity > 0 ? nl->capacity : (int64_t)160 * (N > 0 ? N : 1) + 1024;
  if (nl->auto_size && cap < (int64_t)160 * N + 1024) cap = (int64_t)160 * N + 1024;
  if ((st = reserve(nl, N, NM, cap))) return st;
  const double R = ctx->cfg.rc_rad + ctx->cfg.skin;
  nl->R = R;
  nl->n_atoms = N;
  nl->n_mol = NM;
  nl->stream = s;
  nl->built = true;

  if (N > 0 && N <= SMALL_BUILD_ATOMS && NM <= SMALL_BUILD_MOL) {   // one launch for small systems
    const size_t dyn = sizeof(SmallBuildShared);
    static bool attr_set = false;
    if (!attr_set) {
      FNN_CUDA_TRY(ctx, cudaFuncSetAttribute(k_small_build, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn));
      attr_set = true;
    }
    PredConst pc{R * R, (float)(R * R), (float)R};
    FNN_KERNEL(ctx, "small_build", s);
    k_small_build<<<1, SMALL_NT, dyn, s>>>(*sys, R, pc, nl->capacity, nl->atom_mol, nl->elem, nl->grid, nl->row_ptr,
                                           nl->nbr, nl->shift, nl->perm, nl->inv, nl->tile_elem,
                                           nl->pad_cap / ROW_TILE, nl->pad_cap, nl->meta, ctx->status);
    return check_launch(ctx, "fnn_build_neighbors");
  }
  // cells are bounded by 2N + n_mol + 1 by construction (k_mol_grid caps each structure at max(1, 2n));
  // the structure, cell and row scans each have their own third of the scratch, all cleared by the first
  // kernel
  const int64_t cells_bound = 2LL * N + NM + 1;
  const int64_t third = nl->scan_tmp_len / 3;
  int32_t *tmp_mol = nl->scan_tmp, *tmp_cells = nl->scan_tmp + third, *tmp_rows = nl->scan_tmp + 2 * third;
  int cover_blocks = (NM + 256) / 256 < 256 ? (NM + 256) / 256 : 256;
  {
    FNN_KERNEL(ctx, "check_cover", s);
    k_check_cover<<<cover_blocks, 256, 0, s>>>(*sys, ctx->status, nl->bbox, nl->meta, nl->mol_cells, nl->scan_tmp,
                                               3 * third, nl->meta + META_BAD);
  }
  if (N > 0) {
    int ab = (N + 255) / 256;
    if (ab > 8 * ctx->num_sms) ab = 8 * ctx->num_sms;
    FNN_KERNEL(ctx, "atom_setup", s);
    k_atom_setup<<<ab, 256, 0, s>>>(*sys, nl->atom_mol, nl->elem, nl->bbox, nl->counts, ctx->status,
                                    nl->meta + META_BAD);
  } else {
    FNN_CUDA_TRY(ctx, cudaMemsetAsync(nl->counts, 0, sizeof(int32_t), s));
  }
  // species-sorted order for the networks: needs only the elements, so it runs on the side stream while
  // the cells and pairs are built
  if ((st = side_fork(ctx, s))) return st;
  {
    cudaStream_t ss = ctx->side;
    int nblk = (N + ELEM_NT - 1) / ELEM_NT;
    FNN_CUDA_TRY(ctx, cudaMemsetAsync(nl->inv, 0xff, (size_t)nl->pad_cap * sizeof(int32_t), ss));
    if (nblk > 0) {
      FNN_KERNEL(ctx, "elem_count", ss);
      k_elem_count<<<nblk, ELEM_NT, 0, ss>>>(N, nl->elem, nl->blk_count);
    }
    {
      FNN_KERNEL(ctx, "elem_scan", ss);
      k_elem_scan<<<1, SCAN_NT, 0, ss>>>(nblk, nl->blk_count, nl->meta, nl->tile_elem, nl->pad_cap / ROW_TILE);
    }
    if (nblk > 0) {
      FNN_KERNEL(ctx, "elem_scatter", ss);
      k_elem_scatter<<<nblk, ELEM_NT, 0, ss>>>(N, nl->elem, nl->blk_count, nl->meta, nl->perm, nl->inv);
    }
  }
  {
    FNN_KERNEL(ctx, "mol_grid", s);
    k_mol_grid<<<(NM + 127) / 128, 128, 0, s>>>(*sys, nl->bbox, nl->grid, nl->mol_cells, R, ctx->status,
                                                nl->meta + META_BAD);
  }
  if ((st = exclusive_scan(ctx, nl->mol_cells, nl->mol_cells, NM + 1, nl->meta + META_CELLS, tmp_mol, third, s,
                           nullptr, nullptr, -1, true)))
    return st;
  FNN_CUDA_TRY(ctx, cudaMemsetAsync(nl->cell_count, 0, ((size_t)cells_bound + 1) * sizeof(int32_t), s));
  if (N > 0) {
    int tb = 256, nb = (N + tb - 1) / tb;
    {
      FNN_KERNEL(ctx, "bin", s);
      k_bin<<<nb, tb, 0, s>>>(*sys, nl->grid, nl->mol_cells, nl->atom_mol, nl->cell_of, nl->cell_count, cells_bound);
    }
    // cell starts (over the cells that exist), and the same starts back into the counts as the scatter's cursors
    if ((st = exclusive_scan(ctx, nl->cell_count, nl->cell_start, cells_bound + 1, nullptr, tmp_cells, third, s,
                             nl->meta + META_CELLS, nl->cell_count, -1, true)))
      return st;
    {
      FNN_KERNEL(ctx, "scatter", s);
      k_scatter<<<nb, tb, 0, s>>>(N, nl->cell_of, nl->cell_count, nl->cell_tmp);
    }
    int wb = (int)((cells_bound * 32 + 255) / 256);
    if (wb > 16 * ctx->num_sms) wb = 16 * ctx->num_sms;
    {
      FNN_KERNEL(ctx, "sort_cells", s);
      k_sort_cells<<<wb, 256, 0, s>>>(nl->meta, nl->cell_start, nl->cell_tmp,
                                      reinterpret_cast<const float4 *>(sys->pos), nl->cell_atoms, nl->cell_pos);
    }

    PredConst pc{R * R, (float)(R * R), (float)R};
    int pb = (int)(((int64_t)N * 32 + 255) / 256);
    if (pb > 32 * ctx->num_sms) pb = 32 * ctx->num_sms;
    // up to 32 blocks per SM: a box of ~1000 cells gets four blocks per cell, each staging the stencil
    // and testing a quarter of the centres (47.8 us on the 23,558-atom box, against 52.1 with one block
    // per cell and 54.2 with eight)
    const int cb = (int)(cells_bound < 32 * (int64_t)ctx->num_sms ? cells_bound : 32 * (int64_t)ctx->num_sms);
    {
      FNN_KERNEL(ctx, "pairs_stage", s);
      k_pairs_stage<<<cb > 0 ? cb : 1, CELL_WARPS * 32, 0, s>>>(*sys, nl->grid, nl->mol_cells, nl->atom_mol, nl->cell_of, nl->cell_start,
                                       nl->cell_atoms, nl->cell_pos, pc, nl->counts, nl->stage_nbr, nl->stage_shift,
                                       nl->meta);
    }
    // row pointers; the total is the entry count (FNN_E_CAPACITY beyond the list's capacity)
    if ((st = exclusive_scan(ctx, nl->counts, nl->row_ptr, (int64_t)N + 1, nl->meta + META_NNZ, tmp_rows, third, s,
                             nullptr, nullptr, nl->capacity, true)))
      return st;
    {
      FNN_KERNEL(ctx, "pairs_compact", s);
      k_pairs_compact<<<pb, 256, 0, s>>>(*sys, nl->grid, nl->mol_cells, nl->atom_mol, nl->cell_of, nl->cell_start,
                                         nl->cell_atoms, nl->cell_pos, pc, nl->row_ptr, nl->stage_nbr, nl->stage_shift,
                                         nl->elem, nl->nbr, nl->shift, nl->capacity, nl->meta);
    }
  } else {
    FNN_CUDA_TRY(ctx, cudaMemsetAsync(nl->row_ptr, 0, sizeof(int32_t), s));
  }
  if ((st = side_join(ctx, s))) return st;
  return check_launch(ctx, "fnn_build_neighbors");
}

extern "C" fnn_status fnn_selftest_lookback(fnn_ctx *ctx, int32_t withhold, void *stream) {
  if (!ctx) return FNN_E_INVALID;
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t n = (int64_t)SELFTEST_TILES * SCAN_TILE, ns = 2 * SELFTEST_TILES + 2;
  int32_t *buf = nullptr;
  FNN_CUDA_TRY(ctx, cudaMallocAsync((void **)&buf, (size_t)(n + ns) * sizeof(int32_t), s));
  int32_t *tmp = buf + n;   // 8-byte aligned: n is a multiple of SCAN_TILE
  {
    FNN_KERNEL(ctx, "selftest_fill", s);
    k_selftest_fill<<<8, 256, 0, s>>>(buf, n, tmp, ns);
  }
  {
    FNN_KERNEL(ctx, "scan", s);
    k_scan_single_pass<<<SELFTEST_TILES, SCAN_NT, 0, s>>>(buf, buf, nullptr, n, nullptr, nullptr, -1, tmp,
                                                          ctx->status, withhold != 0);
  }
  if (!withhold) {
    FNN_KERNEL(ctx, "selftest_check", s);
    k_selftest_check<<<8, 256, 0, s>>>(buf, n, ctx->status);
  }
  FNN_CUDA_TRY(ctx, cudaFreeAsync(buf, s));
  return check_launch(ctx, "fnn_selftest_lookback");
}

extern "C" fnn_status fnn_nlist_nnz(fnn_nlist *nl, int64_t *nnz) {
  if (!nl || !nnz) return FNN_E_INVALID;
  if (!nl->built) {
    *nnz = 0;
    return FNN_OK;
  }
  int32_t v = 0;
  FNN_CUDA_TRY(nl->ctx, cudaStreamSynchronize(nl->stream));
  FNN_CUDA_TRY(nl->ctx, cudaMemcpy(&v, nl->row_ptr + nl->n_atoms, sizeof(int32_t), cudaMemcpyDeviceToHost));
  *nnz = v;
  return FNN_OK;
}

extern "C" fnn_status fnn_nlist_export(fnn_nlist *nl, int32_t *row_ptr, int32_t *nbr, int8_t *shift, int64_t cap,
                                       int64_t *nnz) {
  if (!nl || !nnz) return FNN_E_INVALID;
  fnn_status st = fnn_nlist_nnz(nl, nnz);
  if (st) return st;
  if (*nnz > cap || *nnz > nl->capacity) return FNN_E_CAPACITY;
  fnn_ctx *ctx = nl->ctx;
  if (row_ptr)
    FNN_CUDA_TRY(ctx, cudaMemcpy(row_ptr, nl->row_ptr, ((size_t)nl->n_atoms + 1) * sizeof(int32_t),
                                 cudaMemcpyDeviceToHost));
  if (nbr && *nnz > 0)
    FNN_CUDA_TRY(ctx, cudaMemcpy(nbr, nl->nbr, (size_t)*nnz * sizeof(int32_t), cudaMemcpyDeviceToHost));
  if (shift && *nnz > 0) {
    char4 *tmp = (char4 *)malloc((size_t)*nnz * sizeof(char4));
    if (!tmp) return FNN_E_OOM;
    cudaError_t e = cudaMemcpy(tmp, nl->shift, (size_t)*nnz * sizeof(char4), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) {
      free(tmp);
      ctx->last_error = cudaGetErrorString(e);
      return FNN_E_CUDA;
    }
    for (int64_t k = 0; k < *nnz; k++) {
      shift[3 * k] = tmp[k].x;
      shift[3 * k + 1] = tmp[k].y;
      shift[3 * k + 2] = tmp[k].z;
    }
    free(tmp);
  }
  return FNN_OK;
}

// ------------------------------------------------------------------ allocation-free list build
// fnn_build_neighbors_static: the predicate and cell traversal of fnn_build_neighbors in a two-pass
// count/fill form (k_pairs<false>, scan, k_pairs<true>, then k_sort_rows orders rows of at most
// PAIR_STRIDE entries by neighbour element, as k_pairs_compact does), with every scratch array (structure
// grids, cell counts and starts, per-atom cell data, scan partials, status) carved from one file-scope
// device array instead of library allocations.  For callers that may not allocate device memory; sizes
// are capped at FNN_STATIC_MAX_ATOMS atoms and FNN_STATIC_MAX_MOL structures.
#include <mutex>

namespace fnn {
namespace {

constexpr int NS_MAX_ATOMS = FNN_STATIC_MAX_ATOMS;
constexpr int NS_MAX_MOL = FNN_STATIC_MAX_MOL;
constexpr int NS_MAX_CELLS = 2 * NS_MAX_ATOMS + NS_MAX_MOL + 1;   // k_mol_setup caps a structure at 2n cells
constexpr int NS_SCAN_TMP = 64;

struct StaticScratch {
  DevStatus status;
  int32_t meta[META_LEN];
  int32_t scan_tmp[NS_SCAN_TMP];
  MolGrid grid[NS_MAX_MOL];
  int32_t mol_cells[NS_MAX_MOL + 1];
  int32_t atom_mol[NS_MAX_ATOMS];
  int32_t cell_of[NS_MAX_ATOMS];
  int32_t cell_tmp[NS_MAX_ATOMS];
  int32_t cell_atoms[NS_MAX_ATOMS];
  float4 cell_pos[NS_MAX_ATOMS];
  int32_t cell_count[NS_MAX_CELLS + 1];
  int32_t cell_start[NS_MAX_CELLS + 1];
  uint8_t elem[NS_MAX_ATOMS];
};
// the size the header states (423,280 bytes with 8192 atoms and 256 structures)
static_assert(sizeof(StaticScratch) == 423280, "fnn.h states the static scratch size");

// The scratch every call shares (423,280 bytes on every device that loads the library).
static __device__ __align__(256) unsigned char g_nl_scratch[sizeof(StaticScratch)];

constexpr int NS_MAX_DEVICES = 64;
std::mutex g_nl_scratch_mu;
struct ScratchAddr {
  unsigned long long ctx_id = 0;   // driver id of the context the address belongs to (0: none yet)
  StaticScratch *ptr = nullptr;
};
ScratchAddr g_nl_scratch_dev[NS_MAX_DEVICES];

// Unique id of the current thread's CUDA context (0 when the driver cannot say).  Ids are never reused
// within a process, so an address looked up in a context that was since destroyed (cudaDeviceReset) is
// never taken for the new context's.
unsigned long long current_context_id() {
  typedef int (*GetCurrentFn)(void **);
  typedef int (*GetIdFn)(void *, unsigned long long *);
  static GetCurrentFn get_current = nullptr;
  static GetIdFn get_id = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void *f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_current = reinterpret_cast<GetCurrentFn>(f);
    f = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_id = reinterpret_cast<GetIdFn>(f);
    cudaGetLastError();
  });
  void *c = nullptr;
  unsigned long long id = 0;
  if (get_current && get_id && get_current(&c) == 0 && c && get_id(c, &id) == 0) return id;
  return 0;
}

// Device address of the scratch in the current device's context: looked up with cudaGetSymbolAddress
// once per context (a device's first call, and its first call after a context reset), with the device
// current.  When the context id is unavailable the address is looked up on every call.
cudaError_t static_scratch(StaticScratch **out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= NS_MAX_DEVICES) return cudaErrorInvalidDevice;
  if ((e = cudaSetDevice(dev)) != cudaSuccess) return e;   // makes the device's primary context current
  const unsigned long long id = current_context_id();
  std::lock_guard<std::mutex> lock(g_nl_scratch_mu);
  ScratchAddr &a = g_nl_scratch_dev[dev];
  if (id == 0 || a.ctx_id != id || !a.ptr) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_nl_scratch);
    if (e != cudaSuccess) return e;
    a.ptr = reinterpret_cast<StaticScratch *>(p);
    a.ctx_id = id;
  }
  *out = a.ptr;
  return cudaSuccess;
}

cudaError_t scan_in_place(int32_t *data, int64_t n, int32_t *total_dev, int32_t *tmp, cudaStream_t s) {
  int64_t nt = (n + SCAN_TILE - 1) / SCAN_TILE;
  if (n <= 0) return cudaSuccess;
  if (nt > NS_SCAN_TMP) return cudaErrorInvalidValue;
  k_scan_tiles<<<(unsigned)nt, SCAN_NT, 0, s>>>(data, n, tmp);
  k_scan_top<<<1, SCAN_NT, 0, s>>>(tmp, nt, total_dev);
  k_scan_add<<<(unsigned)nt, SCAN_NT, 0, s>>>(data, n, tmp);
  return cudaGetLastError();
}

}  // namespace
}  // namespace fnn

// On a failed step, the work this call already queued is waited for (its error ignored) before the
// error returns, so no kernel of the call still writes the caller's arrays or the shared scratch.
#define FNN_STATIC_TRY(call)                 \
  do {                                       \
    if ((call) != cudaSuccess) {             \
      cudaGetLastError();                    \
      cudaStreamSynchronize(s);              \
      cudaGetLastError();                    \
      return FNN_E_CUDA;                     \
    }                                        \
  } while (0)

extern "C" fnn_status fnn_build_neighbors_static(const fnn_system *sys, double R, int32_t *row_ptr, int32_t *nbr,
                                                 int8_t *shift4, int64_t cap, int64_t *nnz, void *stream) {
  if (!sys || !row_ptr || !nnz || sys->n_atoms < 0 || sys->n_mol < 1 || !sys->mol_offsets || !(R > 0) ||
      cap < 0 || (cap > 0 && (!nbr || !shift4)) || ((uintptr_t)shift4 & 3) != 0 || ((uintptr_t)sys->pos & 15) != 0 ||
      (sys->n_atoms > 0 && (!sys->Z || !sys->pos)) || (sys->pbc && !sys->cell))
    return FNN_E_INVALID;
  *nnz = 0;
  if (sys->n_atoms > NS_MAX_ATOMS || sys->n_mol > NS_MAX_MOL) return FNN_E_CAPACITY;  // beyond the static scratch
  cudaStream_t s = (cudaStream_t)stream;
  StaticScratch *S = nullptr;
  if (static_scratch(&S) != cudaSuccess) {   // nothing queued yet
    cudaGetLastError();
    return FNN_E_CUDA;
  }
  const int N = sys->n_atoms, NM = sys->n_mol;
  const int64_t cells_bound = 2LL * N + NM + 1;

  // clear everything that must start at zero (the array keeps the previous call's contents)
  FNN_STATIC_TRY(cudaMemsetAsync(&S->status, 0, sizeof(DevStatus), s));
  FNN_STATIC_TRY(cudaMemsetAsync(S->meta, 0, sizeof(S->meta), s));
  FNN_STATIC_TRY(cudaMemsetAsync(S->mol_cells, 0, ((size_t)NM + 1) * sizeof(int32_t), s));
  FNN_STATIC_TRY(cudaMemsetAsync(row_ptr, 0, ((size_t)N + 1) * sizeof(int32_t), s));
  if (N > 0) {
    FNN_STATIC_TRY(cudaMemsetAsync(S->atom_mol, 0xff, (size_t)N * sizeof(int32_t), s));
    FNN_STATIC_TRY(cudaMemsetAsync(S->elem, 0, (size_t)N, s));
  }
  k_check_cover<<<1, 256, 0, s>>>(*sys, &S->status, nullptr, nullptr, nullptr, nullptr, 0, S->meta + META_BAD);
  k_mol_setup<<<NM, SETUP_NT, 0, s>>>(*sys, S->grid, S->mol_cells, S->atom_mol, S->elem, R, &S->status,
                                      S->meta + META_BAD);
  FNN_STATIC_TRY(scan_in_place(S->mol_cells, NM + 1, S->meta + META_CELLS, S->scan_tmp, s));
  FNN_STATIC_TRY(cudaMemsetAsync(S->cell_count, 0, ((size_t)cells_bound + 1) * sizeof(int32_t), s));
  FNN_STATIC_TRY(cudaMemsetAsync(S->cell_start, 0, ((size_t)cells_bound + 1) * sizeof(int32_t), s));
  if (N > 0) {
    const int nb = (N + 255) / 256;
    k_bin<<<nb, 256, 0, s>>>(*sys, S->grid, S->mol_cells, S->atom_mol, S->cell_of, S->cell_count, cells_bound);
    FNN_STATIC_TRY(cudaMemcpyAsync(S->cell_start, S->cell_count, ((size_t)cells_bound + 1) * sizeof(int32_t),
                                   cudaMemcpyDeviceToDevice, s));
    FNN_STATIC_TRY(scan_in_place(S->cell_start, cells_bound + 1, nullptr, S->scan_tmp, s));
    FNN_STATIC_TRY(cudaMemcpyAsync(S->cell_count, S->cell_start, ((size_t)cells_bound + 1) * sizeof(int32_t),
                                   cudaMemcpyDeviceToDevice, s));
    k_scatter<<<nb, 256, 0, s>>>(N, S->cell_of, S->cell_count, S->cell_tmp);
    k_sort_cells<<<(int)((cells_bound * 32 + 255) / 256), 256, 0, s>>>(
        S->meta, S->cell_start, S->cell_tmp, reinterpret_cast<const float4 *>(sys->pos), S->cell_atoms, S->cell_pos);
    PredConst pc{R * R, (float)(R * R), (float)R};
    const int pb = (N * 32 + 255) / 256;
    k_pairs<false><<<pb, 256, 0, s>>>(*sys, S->grid, S->mol_cells, S->atom_mol, S->cell_of, S->cell_start,
                                      S->cell_atoms, S->cell_pos, pc, row_ptr, nullptr, nullptr, nullptr, 0, S->meta);
    FNN_STATIC_TRY(scan_in_place(row_ptr, (int64_t)N + 1, nullptr, S->scan_tmp, s));
    k_check_capacity<<<1, 1, 0, s>>>(row_ptr, N, cap, S->meta, &S->status);
    k_pairs<true><<<pb, 256, 0, s>>>(*sys, S->grid, S->mol_cells, S->atom_mol, S->cell_of, S->cell_start,
                                     S->cell_atoms, S->cell_pos, pc, nullptr, row_ptr, nbr,
                                     reinterpret_cast<char4 *>(shift4), cap, S->meta);
    k_sort_rows<<<pb, 256, 0, s>>>(N, row_ptr, S->elem, nbr, reinterpret_cast<char4 *>(shift4), cap);
  }
  FNN_STATIC_TRY(cudaGetLastError());
  int32_t total = 0;
  DevStatus st{};
  FNN_STATIC_TRY(cudaMemcpyAsync(&total, row_ptr + N, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  FNN_STATIC_TRY(cudaMemcpyAsync(&st, &S->status, sizeof(DevStatus), cudaMemcpyDeviceToHost, s));
  FNN_STATIC_TRY(cudaStreamSynchronize(s));
  *nnz = total;
  return (fnn_status)st.code;
}
