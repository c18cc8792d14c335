// Continuous-batching MD service.
//
// One scheduler thread owns a ragged batch of structures resident on the device (positions,
// velocities, forces, neighbour list, per-structure step counters and energy histories).  Every batch
// step is one fnn_energy_forces over the whole batch plus one velocity-Verlet update in which each
// structure advances its own counter, so structures that joined at different times share every
// kernel launch.  Between batch steps the scheduler retires finished structures (results copied to
// the host, waking their pollers) and admits queued requests in arrival order while the estimated
// device memory of the batch stays within the budget; a request larger than the whole budget is
// rejected at submission.  A structure's result does not depend on what else is in the batch:
// structures never interact (section II.A batch index), and each keeps its own list-rebuild schedule
// relative to the skin.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "fnn_internal.cuh"

using namespace fnn;
using Clock = std::chrono::steady_clock;

namespace {

struct Req {
  uint64_t ticket = 0;
  int n = 0;
  std::vector<int32_t> Z;
  std::vector<float> pos4, vel4;   // [n][4]
  float cell[9] = {0};
  uint8_t pbc = 0;
  int n_steps = 0;
  double dt = 0.5;
  Clock::time_point t_submit, t_admit;
};

struct Out {
  std::vector<double> E;
  std::vector<float> pos, vel, F;   // [n][3]
  double latency_ms = 0, queue_ms = 0;
  int n_steps_done = 0;
  fnn_status status = FNN_OK;
};

struct Slot {           // a structure in the device batch
  Req req;
  int offset = 0;       // first atom in the batch arrays
  int step = 0;         // evaluations done
  int since_build = 0;  // evaluations since its list was last rebuilt
  int64_t hist_off = 0; // first entry of its energy history
  fnn_status failed = FNN_OK;   // a device-detected error of this structure alone: it leaves the batch
};

// one copy of a structure's atoms (or history) from a source array into the new layout
struct Seg {
  int64_t src, dst;   // first element in the source and destination
  int32_t n;          // elements
  int32_t from;       // 0: the current batch arrays, 1: the host staging of admitted requests
};

template <typename T>
bool grow(T **p, size_t *cap, size_t need) {
  if (need <= *cap && *p) return true;
  size_t n = need + need / 2 + 64;
  T *q = nullptr;
  if (cudaMalloc(&q, n * sizeof(T)) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (*p) {
    cudaDeviceSynchronize();   // queued work (a result copy on the side stream) may still read the old buffer
    cudaFree(*p);
  }
  *p = q;
  *cap = n;
  return true;
}

}  // namespace

struct fnn_server {
  fnn_ctx *ctx = nullptr;
  size_t budget = 0;
  fnn_precision prec = FNN_BF16;
  int rebuild_every = 10;
  double bytes_per_atom = 0;
  std::thread worker;
  std::mutex mu;
  std::condition_variable cv, cv_done;
  std::deque<Req> pending;
  std::map<uint64_t, Out> done;
  uint64_t next_ticket = 1;
  bool stop = false;
  fnn_status fatal = FNN_OK;
  // statistics
  long long atom_evals = 0, batch_steps = 0, admitted = 0, max_batch_atoms = 0;
  // device batch (double-buffered state for repacking)
  cudaStream_t stream = nullptr;
  fnn_nlist *nl = nullptr;
  std::vector<Slot> active;
  size_t batch_atoms = 0;
  int32_t *Z[2] = {nullptr, nullptr};
  float4 *pos[2] = {nullptr, nullptr}, *vel[2] = {nullptr, nullptr};
  size_t cap_Z[2] = {0, 0}, cap_pos[2] = {0, 0}, cap_vel[2] = {0, 0};
  int cur = 0;
  float *F = nullptr;
  size_t cap_F = 0;
  int32_t *mol_offsets = nullptr, *mol_step = nullptr, *mol_nsteps = nullptr;
  float *cell = nullptr;
  uint8_t *pbc = nullptr;
  double *E = nullptr;
  int64_t *hist_off = nullptr;
  float *mol_dt = nullptr;
  size_t cap_mol = 0, cap_mol2 = 0, cap_mol3 = 0, cap_mol4 = 0, cap_mol5 = 0, cap_mol6 = 0, cap_mol7 = 0, cap_mol8 = 0;
  double *hist = nullptr;        // energy histories of the current layout
  double *hist_buf[2] = {nullptr, nullptr};
  size_t cap_hist[2] = {0, 0};
  // relayout: device staging of admitted requests, segment tables, packed results (device and pinned host)
  int32_t *sZ = nullptr;
  float4 *spos = nullptr, *svel = nullptr;
  size_t cap_sZ = 0, cap_spos = 0, cap_svel = 0;
  Seg *d_seg = nullptr, *h_seg = nullptr;
  size_t cap_seg = 0, cap_hseg = 0;
  int32_t *h_sZ = nullptr;
  float *h_spos = nullptr, *h_svel = nullptr;
  size_t cap_hsZ = 0, cap_hspos = 0, cap_hsvel = 0;
  int64_t *h_mol = nullptr;
  size_t cap_hmol = 0;
  float4 *r_pos = nullptr, *r_vel = nullptr, *h_rpos = nullptr, *h_rvel = nullptr;
  float *r_F = nullptr, *h_rF = nullptr;
  double *r_hist = nullptr, *h_rhist = nullptr;
  size_t cap_rpos = 0, cap_rvel = 0, cap_rF = 0, cap_rhist = 0, cap_hrpos = 0, cap_hrvel = 0, cap_hrF = 0,
         cap_hrhist = 0;
  // results leave on a side stream while the next batch step runs; their segment table has its own buffers
  cudaStream_t cstream = nullptr;
  cudaEvent_t ev_pack = nullptr, ev_ret = nullptr;
  Seg *d_rseg = nullptr, *h_rseg = nullptr;
  size_t cap_rseg = 0, cap_hrseg = 0;
  double host_ms = 0, step_ms = 0;   // worker time in layout changes and in batch steps
  long long failed = 0;              // requests that failed alone (their structure's own error)
  // skin guard: positions at the last rebuild, the batch's largest squared displacement since (device
  // word, and its pinned host copy read after each step)
  float4 *xref = nullptr;
  size_t cap_xref = 0;
  unsigned *d_max_d2 = nullptr;
  float *h_max_d2 = nullptr;
  long long since_any_build = 0, rebuilds = 0, guard_rebuilds = 0;
  std::vector<std::pair<fnn_status, int64_t>> faults;   // device errors of single structures in this step
};

// Index in S->active of the structure a device-detected error belongs to, or -1 when the error concerns
// the whole batch: a non-finite coordinate (info = atom) or energy (info = -(structure + 1)), or an atom
// beyond the AEV kernels' neighbour limits (FNN_E_CAPACITY, info = -(atom + 1)).
static int fault_slot(const fnn_server *S, fnn_status code, int64_t info) {
  int64_t atom = -1;
  if (code == FNN_E_NONFINITE && info < 0) {
    const int64_t m = -info - 1;
    return m < (int64_t)S->active.size() ? (int)m : -1;
  }
  if (code == FNN_E_NONFINITE) atom = info;
  else if (code == FNN_E_CAPACITY && info < 0) atom = -info - 1;
  else return -1;
  int lo = 0, hi = (int)S->active.size();   // last slot whose first atom is <= atom
  if (hi == 0 || atom < S->active[0].offset) return -1;
  while (hi - lo > 1) {
    const int mid = (lo + hi) / 2;
    if (S->active[mid].offset <= atom) lo = mid; else hi = mid;
  }
  return atom < S->active[lo].offset + S->active[lo].req.n ? lo : -1;
}

static double estimate_bytes_per_atom(const fnn_ctx *ctx, fnn_precision prec) {
  const double M = ctx->cfg.n_members;
  const double ws32 = (2.0 * 1008 + M * (256 + 192 + 160 + 192 + 256) + 4 * M + 2) * 4;  // fp32 workspace row
  const double act = (1008 + M * (256 + 192 + 160 + 192 + 256)) * 2 * (prec == FNN_FP32X3 ? 2 : 1);
  const double list = 160 * 8 + 64;
  const double state = 16 * 2 * 2 + 12 + 4;
  return (ws32 + act) * 1.2 + list + state;
}

// relayout of the batch: block per segment; Z, positions and velocities move together
__global__ void k_relayout(const Seg *seg, int nseg, const int32_t *Z0, const float4 *p0, const float4 *v0,
                           const int32_t *Z1, const float4 *p1, const float4 *v1, int32_t *Z, float4 *pos,
                           float4 *vel) {
  for (int k = blockIdx.x; k < nseg; k += gridDim.x) {
    const Seg g = seg[k];
    const int32_t *Zs = g.from ? Z1 : Z0;
    const float4 *ps = g.from ? p1 : p0, *vs = g.from ? v1 : v0;
    for (int i = threadIdx.x; i < g.n; i += blockDim.x) {
      Z[g.dst + i] = Zs[g.src + i];
      pos[g.dst + i] = ps[g.src + i];
      vel[g.dst + i] = vs[g.src + i];
    }
  }
}

// energy histories (doubles) into the new layout
__global__ void k_gather_hist(const Seg *seg, int nseg, const double *src, double *dst) {
  for (int k = blockIdx.x; k < nseg; k += gridDim.x) {
    const Seg g = seg[k];
    for (int i = threadIdx.x; i < g.n; i += blockDim.x) dst[g.dst + i] = src[g.src + i];
  }
}

// finished structures packed for one copy to the host: positions, velocities (float4), forces (3 floats)
__global__ void k_pack_results(const Seg *seg, int nseg, const float4 *pos, const float4 *vel, const float *F,
                               float4 *opos, float4 *ovel, float *oF) {
  for (int k = blockIdx.x; k < nseg; k += gridDim.x) {
    const Seg g = seg[k];
    for (int i = threadIdx.x; i < g.n; i += blockDim.x) {
      opos[g.dst + i] = pos[g.src + i];
      ovel[g.dst + i] = vel[g.src + i];
    }
    for (int i = threadIdx.x; i < 3 * g.n; i += blockDim.x) oF[3 * g.dst + i] = F[3 * g.src + i];
  }
}

template <typename T>
static bool grow_host(T **p, size_t *cap, size_t need) {
  if (need <= *cap && *p) return true;
  size_t n = need + need / 2 + 64;
  T *q = nullptr;
  if (cudaHostAlloc((void **)&q, n * sizeof(T), cudaHostAllocDefault) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (*p) cudaFreeHost(*p);
  *p = q;
  *cap = n;
  return true;
}

// Results of the structures that finished at the last step: packed on the device (batch stream), copied
// to pinned host memory on the side stream, so that the relayout and the next batch step need not wait
// for the host link; finish_retire waits for the copies (ev_ret) while that step runs.
static fnn_status start_retire(fnn_server *S, const std::vector<Slot> &fin) {
  cudaStream_t s = S->stream;
  size_t atoms = 0, hist = 0;
  std::vector<Seg> seg, hseg;
  for (auto &sl : fin) {
    seg.push_back(Seg{sl.offset, (int64_t)atoms, sl.req.n, 0});
    hseg.push_back(Seg{sl.hist_off, (int64_t)hist, sl.req.n_steps, 0});
    atoms += sl.req.n;
    hist += sl.req.n_steps;
  }
  const size_t nseg = seg.size();
  if (!grow(&S->r_pos, &S->cap_rpos, atoms + 1) || !grow(&S->r_vel, &S->cap_rvel, atoms + 1) ||
      !grow(&S->r_F, &S->cap_rF, 3 * atoms + 3) || !grow(&S->r_hist, &S->cap_rhist, hist + 1) ||
      !grow(&S->d_rseg, &S->cap_rseg, 2 * nseg + 2) ||
      !grow_host(&S->h_rpos, &S->cap_hrpos, atoms + 1) || !grow_host(&S->h_rvel, &S->cap_hrvel, atoms + 1) ||
      !grow_host(&S->h_rF, &S->cap_hrF, 3 * atoms + 3) || !grow_host(&S->h_rhist, &S->cap_hrhist, hist + 1) ||
      !grow_host(&S->h_rseg, &S->cap_hrseg, 2 * nseg + 2))
    return FNN_E_OOM;
  memcpy(S->h_rseg, seg.data(), nseg * sizeof(Seg));
  memcpy(S->h_rseg + nseg, hseg.data(), nseg * sizeof(Seg));
  cudaMemcpyAsync(S->d_rseg, S->h_rseg, 2 * nseg * sizeof(Seg), cudaMemcpyHostToDevice, s);
  const int blocks = (int)(nseg < 4096 ? nseg : 4096);
  k_pack_results<<<blocks, 128, 0, s>>>(S->d_rseg, (int)nseg, S->pos[S->cur], S->vel[S->cur], S->F, S->r_pos,
                                         S->r_vel, S->r_F);
  k_gather_hist<<<blocks, 128, 0, s>>>(S->d_rseg + nseg, (int)nseg, S->hist, S->r_hist);
  cudaEventRecord(S->ev_pack, s);
  cudaStreamWaitEvent(S->cstream, S->ev_pack, 0);
  cudaMemcpyAsync(S->h_rpos, S->r_pos, atoms * sizeof(float4), cudaMemcpyDeviceToHost, S->cstream);
  cudaMemcpyAsync(S->h_rvel, S->r_vel, atoms * sizeof(float4), cudaMemcpyDeviceToHost, S->cstream);
  cudaMemcpyAsync(S->h_rF, S->r_F, 3 * atoms * sizeof(float), cudaMemcpyDeviceToHost, S->cstream);
  cudaMemcpyAsync(S->h_rhist, S->r_hist, hist * sizeof(double), cudaMemcpyDeviceToHost, S->cstream);
  cudaEventRecord(S->ev_ret, S->cstream);
  return cudaGetLastError() == cudaSuccess ? FNN_OK : FNN_E_CUDA;
}

// Waits for the result copies of start_retire, then hands each finished structure its output.
static fnn_status finish_retire(fnn_server *S, std::vector<Slot> &fin) {
  if (cudaEventSynchronize(S->ev_ret) != cudaSuccess) {
    cudaGetLastError();
    return FNN_E_CUDA;
  }
  size_t atoms = 0, hist = 0;
  const auto now = Clock::now();
  std::vector<std::pair<uint64_t, Out>> outs;
  outs.reserve(fin.size());
  for (auto &sl : fin) {
    Out o;
    const int n = sl.req.n;
    o.pos.resize(3 * (size_t)n);
    o.vel.resize(3 * (size_t)n);
    o.F.assign(S->h_rF + 3 * atoms, S->h_rF + 3 * (atoms + n));
    o.E.assign(S->h_rhist + hist, S->h_rhist + hist + sl.req.n_steps);
    for (int i = 0; i < n; i++) {
      const float4 p = S->h_rpos[atoms + i], v = S->h_rvel[atoms + i];
      o.pos[3 * i] = p.x; o.pos[3 * i + 1] = p.y; o.pos[3 * i + 2] = p.z;
      o.vel[3 * i] = v.x; o.vel[3 * i + 1] = v.y; o.vel[3 * i + 2] = v.z;
    }
    o.latency_ms = std::chrono::duration<double, std::milli>(now - sl.req.t_submit).count();
    o.queue_ms = std::chrono::duration<double, std::milli>(sl.req.t_admit - sl.req.t_submit).count();
    o.n_steps_done = sl.step;
    atoms += n;
    hist += sl.req.n_steps;
    outs.emplace_back(sl.req.ticket, std::move(o));
  }
  {
    std::lock_guard<std::mutex> lock(S->mu);
    for (auto &po : outs) S->done[po.first] = std::move(po.second);
  }
  S->cv_done.notify_all();
  return FNN_OK;
}

// New layout: survivors (moved on the device), then admitted requests (from pinned host staging), all
// with one segment table and one relayout kernel; per-structure arrays from one pinned block.
static void repack(fnn_server *S, std::vector<Slot> &keep, std::vector<Req> &incoming, fnn_status *err) {
  size_t total = 0, in_atoms = 0;
  for (auto &k : keep) total += k.req.n;
  for (auto &r : incoming) in_atoms += r.n;
  total += in_atoms;
  const int nxt = 1 - S->cur;
  cudaStream_t s = S->stream;
  const size_t nm = keep.size() + incoming.size();
  if (!grow(&S->Z[nxt], &S->cap_Z[nxt], total) || !grow(&S->pos[nxt], &S->cap_pos[nxt], total) ||
      !grow(&S->vel[nxt], &S->cap_vel[nxt], total) || !grow(&S->sZ, &S->cap_sZ, in_atoms + 1) ||
      !grow(&S->spos, &S->cap_spos, in_atoms + 1) || !grow(&S->svel, &S->cap_svel, in_atoms + 1) ||
      !grow_host(&S->h_sZ, &S->cap_hsZ, in_atoms + 1) || !grow_host(&S->h_spos, &S->cap_hspos, 4 * in_atoms + 4) ||
      !grow_host(&S->h_svel, &S->cap_hsvel, 4 * in_atoms + 4) || !grow(&S->d_seg, &S->cap_seg, 2 * nm + 2) ||
      !grow_host(&S->h_seg, &S->cap_hseg, 2 * nm + 2)) {
    *err = FNN_E_OOM;
    return;
  }
  // admitted requests into the pinned staging, one copy each way
  size_t ia = 0;
  for (auto &r : incoming) {
    memcpy(S->h_sZ + ia, r.Z.data(), r.n * sizeof(int32_t));
    memcpy(S->h_spos + 4 * ia, r.pos4.data(), 4 * (size_t)r.n * sizeof(float));
    memcpy(S->h_svel + 4 * ia, r.vel4.data(), 4 * (size_t)r.n * sizeof(float));
    ia += r.n;
    // the structure lives on the device from here on: drop the host copy of its atoms
    std::vector<int32_t>().swap(r.Z);
    std::vector<float>().swap(r.pos4);
    std::vector<float>().swap(r.vel4);
  }
  if (in_atoms) {
    cudaMemcpyAsync(S->sZ, S->h_sZ, in_atoms * sizeof(int32_t), cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(S->spos, S->h_spos, in_atoms * sizeof(float4), cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(S->svel, S->h_svel, in_atoms * sizeof(float4), cudaMemcpyHostToDevice, s);
  }
  size_t off = 0, ioff = 0;
  std::vector<Slot> next;
  next.reserve(nm);
  Seg *seg = S->h_seg;
  std::vector<int> keep_step(keep.size());
  std::vector<int64_t> keep_hist(keep.size());
  for (size_t m = 0; m < keep.size(); m++) {
    Slot &k = keep[m];
    seg[next.size()] = Seg{k.offset, (int64_t)off, k.req.n, 0};
    keep_step[m] = k.step;
    keep_hist[m] = k.hist_off;
    Slot sl = std::move(k);
    sl.offset = (int)off;
    off += sl.req.n;
    next.push_back(std::move(sl));
  }
  for (auto &r : incoming) {
    seg[next.size()] = Seg{(int64_t)ioff, (int64_t)off, r.n, 1};
    Slot sl;
    sl.req = std::move(r);
    sl.offset = (int)off;
    sl.req.t_admit = Clock::now();
    ioff += sl.req.n;
    off += sl.req.n;
    next.push_back(std::move(sl));
  }
  // histories move with their structures into the other buffer of the pair
  int64_t hist_total = 0;
  size_t nh = 0;
  Seg *hseg = seg + nm;
  for (size_t m = 0; m < nm; m++) {
    if (m < keep.size() && keep_step[m] > 0) hseg[nh++] = Seg{keep_hist[m], hist_total, keep_step[m], 0};
    next[m].hist_off = hist_total;
    hist_total += next[m].req.n_steps;
  }
  const int hb = (S->hist == S->hist_buf[0]) ? 1 : 0;
  if (!grow(&S->mol_offsets, &S->cap_mol, nm + 1) || !grow(&S->mol_step, &S->cap_mol2, nm) ||
      !grow(&S->mol_nsteps, &S->cap_mol3, nm) || !grow(&S->cell, &S->cap_mol4, nm * 9) ||
      !grow(&S->pbc, &S->cap_mol5, nm) || !grow(&S->E, &S->cap_mol6, nm) || !grow(&S->hist_off, &S->cap_mol7, nm) ||
      !grow(&S->mol_dt, &S->cap_mol8, nm) || !grow(&S->F, &S->cap_F, 3 * total + 3) ||
      !grow(&S->hist_buf[hb], &S->cap_hist[hb], (size_t)hist_total + 1) ||
      !grow_host(&S->h_mol, &S->cap_hmol, nm * 64 + 64)) {
    *err = FNN_E_OOM;
    return;
  }
  cudaMemcpyAsync(S->d_seg, seg, (nm + nh) * sizeof(Seg), cudaMemcpyHostToDevice, s);
  if (nm) {
    const int blocks = (int)(nm < 4096 ? nm : 4096);
    k_relayout<<<blocks, 128, 0, s>>>(S->d_seg, (int)nm, S->Z[S->cur], S->pos[S->cur], S->vel[S->cur], S->sZ, S->spos,
                                      S->svel, S->Z[nxt], S->pos[nxt], S->vel[nxt]);
  }
  double *new_hist = S->hist_buf[hb];
  if (nh) {
    const int blocks = (int)(nh < 4096 ? nh : 4096);
    k_gather_hist<<<blocks, 128, 0, s>>>(S->d_seg + nm, (int)nh, S->hist, new_hist);
  }
  // per-structure arrays from one pinned block
  char *hm = reinterpret_cast<char *>(S->h_mol);
  int32_t *mo = reinterpret_cast<int32_t *>(hm);
  int32_t *st = mo + (nm + 1);
  int32_t *ns = st + nm;
  float *ce = reinterpret_cast<float *>(ns + nm);
  float *dts = ce + 9 * nm;
  int64_t *ho = reinterpret_cast<int64_t *>(hm + (((char *)(dts + nm) - hm + 7) & ~(size_t)7));
  uint8_t *pb = reinterpret_cast<uint8_t *>(ho + nm);
  for (size_t m = 0; m < nm; m++) {
    mo[m] = next[m].offset;
    st[m] = next[m].step;
    ns[m] = next[m].req.n_steps;
    memcpy(&ce[9 * m], next[m].req.cell, 9 * sizeof(float));
    dts[m] = (float)next[m].req.dt;
    ho[m] = next[m].hist_off;
    pb[m] = next[m].req.pbc;
  }
  mo[nm] = (int32_t)total;
  cudaMemcpyAsync(S->mol_offsets, mo, (nm + 1) * sizeof(int32_t), cudaMemcpyHostToDevice, s);
  cudaMemcpyAsync(S->mol_step, st, nm * sizeof(int32_t), cudaMemcpyHostToDevice, s);
  cudaMemcpyAsync(S->mol_nsteps, ns, nm * sizeof(int32_t), cudaMemcpyHostToDevice, s);
  cudaMemcpyAsync(S->cell, ce, nm * 9 * sizeof(float), cudaMemcpyHostToDevice, s);
  cudaMemcpyAsync(S->mol_dt, dts, nm * sizeof(float), cudaMemcpyHostToDevice, s);
  cudaMemcpyAsync(S->hist_off, ho, nm * sizeof(int64_t), cudaMemcpyHostToDevice, s);
  cudaMemcpyAsync(S->pbc, pb, nm, cudaMemcpyHostToDevice, s);
  // the pinned blocks are rewritten only after the next stream synchronisation (end of the batch step)
  S->hist = new_hist;
  S->cur = nxt;
  S->active = std::move(next);
  S->batch_atoms = total;
  for (auto &sl : S->active) sl.since_build = 0;   // the batch layout changed: every list is rebuilt
  if (cudaGetLastError() != cudaSuccess) *err = FNN_E_CUDA;
}

// one batch step: (re)build lists, energy + forces for every structure, record energies, advance
static fnn_status serve_step(fnn_server *S) {
  fnn_ctx *ctx = S->ctx;
  const int nm = (int)S->active.size();
  fnn_system sys{(int32_t)S->batch_atoms, nm, S->mol_offsets, S->Z[S->cur], reinterpret_cast<float *>(S->pos[S->cur]),
                 S->cell, S->pbc};
  bool rebuild = false, due = false;
  for (auto &sl : S->active)
    if (sl.since_build == 0 || sl.since_build >= S->rebuild_every) due = true;
  // skin guard: an atom of some structure moved more than skin/2 since the last rebuild (the largest
  // displacement of the batch, read back with the previous step)
  const double hs = 0.5 * ctx->cfg.skin;
  const bool moved = S->since_any_build > 0 && (double)*S->h_max_d2 > hs * hs;
  rebuild = due || moved;
  fnn_status st;
  if (!grow(&S->xref, &S->cap_xref, S->batch_atoms + 1)) return FNN_E_OOM;
  // the list and (through its padded row count) every network workspace grow geometrically with the
  // batch, so a batch that keeps growing does not reallocate gigabytes at every step
  if (sys.n_atoms > S->nl->atom_cap || nm > S->nl->mol_cap) {
    const int32_t na = 2 * sys.n_atoms, nmol = 2 * nm;
    if ((st = fnn_nlist_reserve(S->nl, na, nmol, (int64_t)160 * na + 1024))) return st;
  }
  if (rebuild) {
    // a list larger than its capacity is regrown and rebuilt before any force is computed
    for (int attempt = 0; attempt < 2; attempt++) {
      if ((st = fnn_build_neighbors(ctx, &sys, S->nl, S->stream))) return st;
      int64_t info = 0;
      st = fnn_sync(ctx, S->stream, &info);
      if (st == FNN_E_CAPACITY && info > 0 && attempt == 0) {
        if ((st = fnn_nlist_reserve(S->nl, sys.n_atoms, nm, info + info / 4))) return st;
        continue;
      }
      if (st && fault_slot(S, st, info) >= 0) {   // one structure's own error: the others go on
        S->faults.emplace_back(st, info);
        st = FNN_OK;
      }
      if (st) return st;
      break;
    }
    for (auto &sl : S->active) sl.since_build = 0;
    S->since_any_build = 0;
    S->rebuilds++;
    if (!due) S->guard_rebuilds++;
    if ((st = launch_md_ref(ctx, sys.n_atoms, S->pos[S->cur], S->xref, S->stream))) return st;
    FNN_CUDA_TRY(ctx, cudaMemsetAsync(S->d_max_d2, 0, sizeof(unsigned), S->stream));
  }
  if ((st = fnn_energy_forces(ctx, &sys, S->nl, S->prec, S->E, S->F, nullptr, S->stream))) return st;
  if ((st = launch_record_energy(ctx, nm, S->E, S->mol_step, S->mol_nsteps, S->hist_off, S->hist, 0, 0, S->stream)))
    return st;
  MdUpdate u;
  u.mol_step = S->mol_step;
  u.mol_nsteps = S->mol_nsteps;
  u.mol_dt = S->mol_dt;
  u.xref = S->xref;
  u.max_d2 = S->d_max_d2;
  if ((st = launch_md_update(ctx, S->nl, (int)S->batch_atoms, S->pos[S->cur], S->vel[S->cur], S->F, u, S->stream)))
    return st;
  if ((st = launch_advance_steps(ctx, nm, S->mol_step, nullptr, S->stream))) return st;
  FNN_CUDA_TRY(ctx, cudaMemcpyAsync(S->h_max_d2, S->d_max_d2, sizeof(unsigned), cudaMemcpyDeviceToHost, S->stream));
  for (auto &sl : S->active) {
    sl.step++;
    sl.since_build++;
  }
  S->since_any_build++;
  return FNN_OK;
}

static void fail_all(fnn_server *S, fnn_status err) {
  std::lock_guard<std::mutex> lock(S->mu);
  S->fatal = err;
  for (auto &sl : S->active) {
    Out o;
    o.status = err;
    S->done[sl.req.ticket] = std::move(o);
  }
  S->active.clear();
  S->cv_done.notify_all();
}

static void worker_main(fnn_server *S) {
  cudaSetDevice(S->ctx->device);
  std::vector<Slot> fin;   // finished at the last batch step, results not yet taken
  for (;;) {
    std::vector<Req> incoming;
    {
      std::unique_lock<std::mutex> lock(S->mu);
      S->cv.wait(lock, [&] { return S->stop || !S->pending.empty() || !S->active.empty() || !fin.empty(); });
      if (S->stop && S->active.empty() && S->pending.empty() && fin.empty()) break;
      // admit in arrival order while the batch fits the budget
      double in_use = 0;
      for (auto &sl : S->active)
        if (sl.step < sl.req.n_steps) in_use += sl.req.n * S->bytes_per_atom;
      while (!S->pending.empty() && in_use + S->pending.front().n * S->bytes_per_atom <= (double)S->budget) {
        in_use += S->pending.front().n * S->bytes_per_atom;
        incoming.push_back(std::move(S->pending.front()));
        S->pending.pop_front();
      }
      S->admitted += (long long)incoming.size();
    }
    const auto t0 = Clock::now();
    // structures with nothing to evaluate finish at once
    for (auto it = incoming.begin(); it != incoming.end();) {
      if (it->n_steps <= 0) {
        Out o;
        o.latency_ms = std::chrono::duration<double, std::milli>(Clock::now() - it->t_submit).count();
        {
          std::lock_guard<std::mutex> lock(S->mu);
          S->done[it->ticket] = std::move(o);
        }
        S->cv_done.notify_all();
        it = incoming.erase(it);
      } else {
        ++it;
      }
    }
    fnn_status err = FNN_OK;
    std::vector<Slot> keep;
    const bool changed = !incoming.empty() ||
                         std::any_of(S->active.begin(), S->active.end(), [](const Slot &sl) {
                           return sl.step >= sl.req.n_steps || sl.failed != FNN_OK;
                         });
    if (changed) {
      std::vector<std::pair<uint64_t, Out>> failed_out;
      for (auto &sl : S->active) {
        if (sl.failed != FNN_OK) {   // its own error: its ticket fails, nothing of it is copied back
          Out o;
          o.status = sl.failed;
          o.latency_ms = std::chrono::duration<double, std::milli>(Clock::now() - sl.req.t_submit).count();
          o.n_steps_done = sl.step;
          failed_out.emplace_back(sl.req.ticket, std::move(o));
          continue;
        }
        (sl.step >= sl.req.n_steps ? fin : keep).push_back(std::move(sl));
      }
      S->active.clear();
      if (!failed_out.empty()) {
        {
          std::lock_guard<std::mutex> lock(S->mu);
          S->failed += (long long)failed_out.size();
          for (auto &po : failed_out) S->done[po.first] = std::move(po.second);
        }
        S->cv_done.notify_all();
      }
    }
    if (!fin.empty()) err = start_retire(S, fin);
    const bool retiring = !fin.empty() && err == FNN_OK;
    if (err == FNN_OK && changed) repack(S, keep, incoming, &err);
    const auto t1 = Clock::now();
    // the finished structures' results are handed out while the batch step runs on the device
    const bool stepping = err == FNN_OK && !S->active.empty();
    if (stepping) err = serve_step(S);
    if (retiring) {
      const fnn_status rs = finish_retire(S, fin);
      if (rs == FNN_OK) fin.clear();
      else if (err == FNN_OK) err = rs;
    }
    if (stepping) {
      if (err == FNN_OK) {
        int64_t info = 0;
        err = fnn_sync(S->ctx, S->stream, &info);
        if (err != FNN_OK && fault_slot(S, err, info) >= 0) {
          S->faults.emplace_back(err, info);
          err = FNN_OK;
        }
      }
      // structures with their own error leave the batch at the next layout change; the step's results of
      // every other structure stand (structures never interact)
      for (auto &f : S->faults) {
        const int k = fault_slot(S, f.first, f.second);
        if (k >= 0 && S->active[k].failed == FNN_OK) S->active[k].failed = f.first;
      }
      S->faults.clear();
      std::lock_guard<std::mutex> lock(S->mu);
      S->batch_steps++;
      S->atom_evals += (long long)S->batch_atoms;
      if ((long long)S->batch_atoms > S->max_batch_atoms) S->max_batch_atoms = (long long)S->batch_atoms;
    }
    const auto t2 = Clock::now();
    {
      std::lock_guard<std::mutex> lock(S->mu);
      S->host_ms += std::chrono::duration<double, std::milli>(t1 - t0).count();
      S->step_ms += std::chrono::duration<double, std::milli>(t2 - t1).count();
    }
    if (err != FNN_OK) {
      // every structure still waiting for its result fails (tickets survive a move of their slot)
      if (S->active.empty())
        for (auto &sl : keep) S->active.push_back(std::move(sl));
      for (auto &sl : fin) S->active.push_back(std::move(sl));
      fin.clear();
      fail_all(S, err);
    }
  }
}

extern "C" fnn_status fnn_serve_create(fnn_server **out, fnn_ctx *ctx, size_t hbm_budget_bytes, fnn_precision prec,
                                       int32_t rebuild_every) {
  if (!out || !ctx || hbm_budget_bytes == 0 || rebuild_every < 1 ||
      (prec != FNN_FP32 && prec != FNN_BF16 && prec != FNN_FP32X3 && prec != FNN_BF16_FUSED))
    return FNN_E_INVALID;
  if (!ctx->has_weights) return FNN_E_STATE;
  fnn_server *S = new fnn_server();
  S->ctx = ctx;
  S->budget = hbm_budget_bytes;
  S->prec = prec;
  S->rebuild_every = rebuild_every;
  S->bytes_per_atom = estimate_bytes_per_atom(ctx, prec);
  if (cudaStreamCreateWithFlags(&S->stream, cudaStreamNonBlocking) != cudaSuccess) {
    delete S;
    return FNN_E_CUDA;
  }
  if (cudaStreamCreateWithFlags(&S->cstream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&S->ev_pack, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&S->ev_ret, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    if (S->ev_pack) cudaEventDestroy(S->ev_pack);
    if (S->cstream) cudaStreamDestroy(S->cstream);
    cudaStreamDestroy(S->stream);
    delete S;
    return FNN_E_CUDA;
  }
  fnn_status st = fnn_nlist_create(ctx, &S->nl, 0);
  if (!st && (cudaMalloc((void **)&S->d_max_d2, 256) != cudaSuccess ||
              cudaHostAlloc((void **)&S->h_max_d2, 64, cudaHostAllocDefault) != cudaSuccess)) {
    cudaGetLastError();
    if (S->d_max_d2) cudaFree(S->d_max_d2);
    fnn_nlist_destroy(S->nl);
    st = FNN_E_OOM;
  }
  if (!st) {
    *S->h_max_d2 = 0.f;
    cudaMemset(S->d_max_d2, 0, 256);
  }
  if (st) {
    cudaEventDestroy(S->ev_pack);
    cudaEventDestroy(S->ev_ret);
    cudaStreamDestroy(S->cstream);
    cudaStreamDestroy(S->stream);
    delete S;
    return st;
  }
  S->worker = std::thread(worker_main, S);
  *out = S;
  return FNN_OK;
}

extern "C" fnn_status fnn_serve_submit(fnn_server *S, const fnn_request *q, uint64_t *ticket) {
  if (!S || !q || !ticket || q->n_atoms < 0 || (q->n_atoms > 0 && (!q->Z || !q->pos)) || !(q->dt_fs > 0))
    return FNN_E_INVALID;
  if (q->n_steps < 0) return FNN_E_INVALID;
  if (q->n_atoms * S->bytes_per_atom > (double)S->budget) return FNN_E_OOM;   // alone it exceeds the budget
  // what the device would reject for the whole batch is rejected here, for this request alone
  for (int i = 0; i < q->n_atoms; i++) {
    if (element_of(q->Z[i]) < 0) return FNN_E_SPECIES;
    for (int a = 0; a < 3; a++)
      if (!std::isfinite(q->pos[3 * i + a]) || (q->vel && !std::isfinite(q->vel[3 * i + a]))) return FNN_E_NONFINITE;
  }
  if (q->cell) {
    const float *c = q->cell;
    const double R = S->ctx->cfg.rc_rad + S->ctx->cfg.skin;
    const bool ortho = c[1] == 0.f && c[2] == 0.f && c[3] == 0.f && c[5] == 0.f && c[6] == 0.f && c[7] == 0.f;
    if (!ortho || !((double)c[0] > 2 * R) || !((double)c[4] > 2 * R) || !((double)c[8] > 2 * R)) return FNN_E_CELL;
  }
  Req r;
  r.n = q->n_atoms;
  r.Z.assign(q->Z, q->Z + q->n_atoms);
  r.pos4.resize(4 * (size_t)r.n);
  r.vel4.assign(4 * (size_t)r.n, 0.f);
  for (int i = 0; i < r.n; i++) {
    for (int a = 0; a < 3; a++) {
      r.pos4[4 * i + a] = q->pos[3 * i + a];
      if (q->vel) r.vel4[4 * i + a] = q->vel[3 * i + a];
    }
    r.pos4[4 * i + 3] = 0.f;
  }
  if (q->cell) {
    memcpy(r.cell, q->cell, 9 * sizeof(float));
    r.pbc = 1;
  }
  r.n_steps = q->n_steps;
  r.dt = q->dt_fs;
  r.t_submit = Clock::now();
  {
    std::lock_guard<std::mutex> lock(S->mu);
    if (S->stop) return FNN_E_STATE;
    r.ticket = S->next_ticket++;
    *ticket = r.ticket;
    S->pending.push_back(std::move(r));
  }
  S->cv.notify_one();
  return FNN_OK;
}

extern "C" fnn_status fnn_serve_poll(fnn_server *S, uint64_t ticket, fnn_result *res, int64_t timeout_us) {
  if (!S || !res) return FNN_E_INVALID;
  std::unique_lock<std::mutex> lock(S->mu);
  auto ready = [&] { return S->done.count(ticket) > 0; };
  if (!ready()) {
    if (timeout_us <= 0) return FNN_PENDING;
    if (!S->cv_done.wait_for(lock, std::chrono::microseconds(timeout_us), ready)) return FNN_PENDING;
  }
  Out o = std::move(S->done[ticket]);
  S->done.erase(ticket);
  lock.unlock();
  if (o.status != FNN_OK) return o.status;
  const int n = (int)o.pos.size() / 3;
  if (res->energies && !o.E.empty()) memcpy(res->energies, o.E.data(), o.E.size() * sizeof(double));
  if (res->pos && n) memcpy(res->pos, o.pos.data(), o.pos.size() * sizeof(float));
  if (res->vel && n) memcpy(res->vel, o.vel.data(), o.vel.size() * sizeof(float));
  if (res->forces && n) memcpy(res->forces, o.F.data(), o.F.size() * sizeof(float));
  res->latency_ms = o.latency_ms;
  res->queue_ms = o.queue_ms;
  res->n_steps_done = o.n_steps_done;
  return FNN_OK;
}

extern "C" fnn_status fnn_serve_stats(fnn_server *S, fnn_serve_counters *st) {
  if (!S || !st) return FNN_E_INVALID;
  std::lock_guard<std::mutex> lock(S->mu);
  st->atom_evals = S->atom_evals;
  st->batch_steps = S->batch_steps;
  st->admitted = S->admitted;
  st->max_batch_atoms = S->max_batch_atoms;
  st->pending = (int64_t)S->pending.size();
  st->bytes_per_atom = S->bytes_per_atom;
  st->host_ms = S->host_ms;
  st->step_ms = S->step_ms;
  st->failed = S->failed;
  st->rebuilds = S->rebuilds;
  st->guard_rebuilds = S->guard_rebuilds;
  return S->fatal;
}

extern "C" fnn_status fnn_serve_destroy(fnn_server *S) {
  if (!S) return FNN_E_INVALID;
  {
    std::lock_guard<std::mutex> lock(S->mu);
    S->stop = true;
  }
  S->cv.notify_all();
  if (S->worker.joinable()) S->worker.join();
  cudaStreamSynchronize(S->stream);
  cudaStreamSynchronize(S->cstream);
  for (int b = 0; b < 2; b++) {
    if (S->Z[b]) cudaFree(S->Z[b]);
    if (S->pos[b]) cudaFree(S->pos[b]);
    if (S->vel[b]) cudaFree(S->vel[b]);
  }
  void *ptrs[] = {S->F, S->mol_offsets, S->mol_step, S->mol_nsteps, S->cell, S->pbc, S->E, S->hist_off,
                  S->hist_buf[0], S->hist_buf[1], S->mol_dt, S->sZ, S->spos, S->svel, S->d_seg,
                  S->d_rseg, S->r_pos, S->r_vel, S->r_F, S->r_hist, S->xref, S->d_max_d2};
  for (void *p : ptrs)
    if (p) cudaFree(p);
  void *hptrs[] = {S->h_seg,  S->h_rseg, S->h_sZ,   S->h_spos,  S->h_svel,
                   S->h_mol,  S->h_rpos, S->h_rvel, S->h_rF,    S->h_rhist, S->h_max_d2};
  for (void *p : hptrs)
    if (p) cudaFreeHost(p);
  if (S->nl) fnn_nlist_destroy(S->nl);
  cudaEventDestroy(S->ev_pack);
  cudaEventDestroy(S->ev_ret);
  cudaStreamDestroy(S->cstream);
  cudaStreamDestroy(S->stream);
  delete S;
  return FNN_OK;
}
