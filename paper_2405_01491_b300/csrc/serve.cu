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
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "fnn_internal.cuh"

namespace fnn {
fnn_status launch_vv(fnn_ctx *ctx, const fnn_nlist *nl, int n, float4 *pos, float4 *vel, const float *F,
                     const int32_t *mol_step, const int32_t *mol_nsteps, const float *mol_dt, int step, int nsteps,
                     double dt, cudaStream_t s);
fnn_status launch_record_energy(fnn_ctx *ctx, int n_mol, const double *E, const int32_t *mol_step,
                                const int32_t *mol_nsteps, const int64_t *hist_off, double *hist, int step,
                                int64_t stride, cudaStream_t s);
fnn_status launch_advance_steps(fnn_ctx *ctx, int n_mol, int32_t *mol_step, cudaStream_t s);
}  // namespace fnn

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
  if (*p) cudaFree(*p);
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
  // pinned staging for the host copies
  std::vector<float> host_tmp;
};

static double estimate_bytes_per_atom(const fnn_ctx *ctx, fnn_precision prec) {
  const double M = ctx->cfg.n_members;
  const double ws32 = (2.0 * 1008 + M * (256 + 192 + 160 + 192 + 256) + 4 * M + 2) * 4;  // fp32 workspace row
  const double act = (1008 + M * (256 + 192 + 160 + 192 + 256)) * 2 * (prec == FNN_FP32X3 ? 2 : 1);
  const double list = 160 * 8 + 64;
  const double state = 16 * 2 * 2 + 12 + 4;
  return (ws32 + act) * 1.2 + list + state;
}

static fnn_status serve_step(fnn_server *S);

static void repack(fnn_server *S, std::vector<Slot> &keep, std::vector<Req> &incoming, fnn_status *err) {
  // new layout: survivors (copied on the device), then new structures (copied from the host)
  size_t total = 0;
  for (auto &k : keep) total += k.req.n;
  for (auto &r : incoming) total += r.n;
  const int nxt = 1 - S->cur;
  if (!grow(&S->Z[nxt], &S->cap_Z[nxt], total) || !grow(&S->pos[nxt], &S->cap_pos[nxt], total) ||
      !grow(&S->vel[nxt], &S->cap_vel[nxt], total)) {
    *err = FNN_E_OOM;
    return;
  }
  cudaStream_t s = S->stream;
  size_t off = 0;
  std::vector<Slot> next;
  for (auto &k : keep) {
    cudaMemcpyAsync(S->Z[nxt] + off, S->Z[S->cur] + k.offset, k.req.n * sizeof(int32_t), cudaMemcpyDeviceToDevice, s);
    cudaMemcpyAsync(S->pos[nxt] + off, S->pos[S->cur] + k.offset, k.req.n * sizeof(float4), cudaMemcpyDeviceToDevice, s);
    cudaMemcpyAsync(S->vel[nxt] + off, S->vel[S->cur] + k.offset, k.req.n * sizeof(float4), cudaMemcpyDeviceToDevice, s);
    Slot sl = k;
    sl.offset = (int)off;
    next.push_back(sl);
    off += k.req.n;
  }
  for (auto &r : incoming) {
    cudaMemcpyAsync(S->Z[nxt] + off, r.Z.data(), r.n * sizeof(int32_t), cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(S->pos[nxt] + off, r.pos4.data(), r.n * sizeof(float4), cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(S->vel[nxt] + off, r.vel4.data(), r.n * sizeof(float4), cudaMemcpyHostToDevice, s);
    Slot sl;
    sl.req = std::move(r);
    sl.offset = (int)off;
    sl.req.t_admit = Clock::now();
    next.push_back(std::move(sl));
    off += next.back().req.n;
  }
  // per-structure arrays
  const size_t nm = next.size();
  if (!grow(&S->mol_offsets, &S->cap_mol, nm + 1) || !grow(&S->mol_step, &S->cap_mol2, nm) ||
      !grow(&S->mol_nsteps, &S->cap_mol3, nm) || !grow(&S->cell, &S->cap_mol4, nm * 9) ||
      !grow(&S->pbc, &S->cap_mol5, nm) || !grow(&S->E, &S->cap_mol6, nm) || !grow(&S->hist_off, &S->cap_mol7, nm) ||
      !grow(&S->mol_dt, &S->cap_mol8, nm) || !grow(&S->F, &S->cap_F, 3 * total + 3)) {
    *err = FNN_E_OOM;
    return;
  }
  std::vector<int32_t> mo(nm + 1), st(nm), ns(nm);
  std::vector<float> ce(nm * 9);
  std::vector<uint8_t> pb(nm);
  std::vector<int64_t> ho(nm);
  std::vector<float> dts(nm);
  int64_t hist_total = 0;
  for (size_t m = 0; m < nm; m++) {
    mo[m] = next[m].offset;
    st[m] = next[m].step;
    ns[m] = next[m].req.n_steps;
    memcpy(&ce[9 * m], next[m].req.cell, 9 * sizeof(float));
    pb[m] = next[m].req.pbc;
    dts[m] = (float)next[m].req.dt;
    ho[m] = hist_total;
    hist_total += next[m].req.n_steps;
  }
  mo[nm] = (int32_t)total;
  // histories move with their structures into the other buffer of the pair (grow-only, no frees here)
  double *old_hist = S->hist;
  const int hb = (S->hist == S->hist_buf[0]) ? 1 : 0;
  if (!grow(&S->hist_buf[hb], &S->cap_hist[hb], (size_t)hist_total + 1)) {
    *err = FNN_E_OOM;
    return;
  }
  double *new_hist = S->hist_buf[hb];
  for (size_t m = 0; m < keep.size(); m++)
    if (keep[m].step > 0)
      cudaMemcpyAsync(new_hist + ho[m], old_hist + keep[m].hist_off, keep[m].step * sizeof(double),
                      cudaMemcpyDeviceToDevice, s);
  for (size_t m = 0; m < nm; m++) next[m].hist_off = ho[m];
  cudaMemcpyAsync(S->mol_offsets, mo.data(), (nm + 1) * sizeof(int32_t), cudaMemcpyHostToDevice, s);
  cudaMemcpyAsync(S->mol_step, st.data(), nm * sizeof(int32_t), cudaMemcpyHostToDevice, s);
  cudaMemcpyAsync(S->mol_nsteps, ns.data(), nm * sizeof(int32_t), cudaMemcpyHostToDevice, s);
  cudaMemcpyAsync(S->cell, ce.data(), nm * 9 * sizeof(float), cudaMemcpyHostToDevice, s);
  cudaMemcpyAsync(S->pbc, pb.data(), nm, cudaMemcpyHostToDevice, s);
  cudaMemcpyAsync(S->hist_off, ho.data(), nm * sizeof(int64_t), cudaMemcpyHostToDevice, s);
  cudaMemcpyAsync(S->mol_dt, dts.data(), nm * sizeof(float), cudaMemcpyHostToDevice, s);
  cudaStreamSynchronize(s);   // host vectors above must outlive their copies
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
  bool rebuild = false;
  for (auto &sl : S->active)
    if (sl.since_build == 0 || sl.since_build >= S->rebuild_every) rebuild = true;
  fnn_status st;
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
      if (st) return st;
      break;
    }
    for (auto &sl : S->active) sl.since_build = 0;
  }
  if ((st = fnn_energy_forces(ctx, &sys, S->nl, S->prec, S->E, S->F, nullptr, S->stream))) return st;
  if ((st = launch_record_energy(ctx, nm, S->E, S->mol_step, S->mol_nsteps, S->hist_off, S->hist, 0, 0, S->stream)))
    return st;
  if ((st = launch_vv(ctx, S->nl, (int)S->batch_atoms, S->pos[S->cur], S->vel[S->cur], S->F, S->mol_step,
                      S->mol_nsteps, S->mol_dt, 0, 0, 0.0, S->stream)))
    return st;
  if ((st = launch_advance_steps(ctx, nm, S->mol_step, S->stream))) return st;
  for (auto &sl : S->active) {
    sl.step++;
    sl.since_build++;
  }
  return FNN_OK;
}

static void retire(fnn_server *S, std::vector<Slot> &finished) {
  cudaStream_t s = S->stream;
  for (auto &sl : finished) {
    Out o;
    const int n = sl.req.n;
    std::vector<float4> p4(n), v4(n);
    o.F.resize(3 * (size_t)n);
    o.E.resize(sl.req.n_steps);
    cudaMemcpyAsync(p4.data(), S->pos[S->cur] + sl.offset, n * sizeof(float4), cudaMemcpyDeviceToHost, s);
    cudaMemcpyAsync(v4.data(), S->vel[S->cur] + sl.offset, n * sizeof(float4), cudaMemcpyDeviceToHost, s);
    cudaMemcpyAsync(o.F.data(), S->F + 3 * (size_t)sl.offset, 3 * (size_t)n * sizeof(float), cudaMemcpyDeviceToHost, s);
    if (sl.req.n_steps > 0)
      cudaMemcpyAsync(o.E.data(), S->hist + sl.hist_off, sl.req.n_steps * sizeof(double), cudaMemcpyDeviceToHost, s);
    cudaStreamSynchronize(s);
    o.pos.resize(3 * (size_t)n);
    o.vel.resize(3 * (size_t)n);
    for (int i = 0; i < n; i++) {
      o.pos[3 * i] = p4[i].x; o.pos[3 * i + 1] = p4[i].y; o.pos[3 * i + 2] = p4[i].z;
      o.vel[3 * i] = v4[i].x; o.vel[3 * i + 1] = v4[i].y; o.vel[3 * i + 2] = v4[i].z;
    }
    const auto now = Clock::now();
    o.latency_ms = std::chrono::duration<double, std::milli>(now - sl.req.t_submit).count();
    o.queue_ms = std::chrono::duration<double, std::milli>(sl.req.t_admit - sl.req.t_submit).count();
    o.n_steps_done = sl.step;
    std::lock_guard<std::mutex> lock(S->mu);
    S->done[sl.req.ticket] = std::move(o);
  }
  S->cv_done.notify_all();
}

static void worker_main(fnn_server *S) {
  cudaSetDevice(S->ctx->device);
  for (;;) {
    std::vector<Req> incoming;
    {
      std::unique_lock<std::mutex> lock(S->mu);
      S->cv.wait(lock, [&] { return S->stop || !S->pending.empty() || !S->active.empty(); });
      if (S->stop && S->active.empty() && S->pending.empty()) break;
      // admit in arrival order while the batch fits the budget
      double in_use = 0;
      for (auto &sl : S->active) in_use += sl.req.n * S->bytes_per_atom;
      while (!S->pending.empty() && in_use + S->pending.front().n * S->bytes_per_atom <= (double)S->budget) {
        in_use += S->pending.front().n * S->bytes_per_atom;
        incoming.push_back(std::move(S->pending.front()));
        S->pending.pop_front();
      }
    }
    // structures with nothing to evaluate finish at once
    std::vector<Slot> finished;
    for (auto it = incoming.begin(); it != incoming.end();) {
      if (it->n_steps <= 0) {
        Slot sl;
        sl.req = std::move(*it);
        sl.req.t_admit = Clock::now();
        finished.push_back(std::move(sl));
        it = incoming.erase(it);
      } else {
        ++it;
      }
    }
    if (!finished.empty()) {
      std::vector<Slot> none;
      for (auto &sl : finished) {
        std::lock_guard<std::mutex> lock(S->mu);
        Out o;
        o.latency_ms = std::chrono::duration<double, std::milli>(Clock::now() - sl.req.t_submit).count();
        S->done[sl.req.ticket] = std::move(o);
      }
      S->cv_done.notify_all();
    }
    fnn_status err = FNN_OK;
    if (!incoming.empty()) {
      std::vector<Slot> keep = S->active;
      repack(S, keep, incoming, &err);
      std::lock_guard<std::mutex> lock(S->mu);
      S->admitted += (long long)incoming.size();
    }
    if (err == FNN_OK && !S->active.empty()) {
      err = serve_step(S);
      if (err == FNN_OK) {
        int64_t info = 0;
        err = fnn_sync(S->ctx, S->stream, &info);
      }
      std::lock_guard<std::mutex> lock(S->mu);
      S->batch_steps++;
      S->atom_evals += (long long)S->batch_atoms;
      if ((long long)S->batch_atoms > S->max_batch_atoms) S->max_batch_atoms = (long long)S->batch_atoms;
    }
    if (err != FNN_OK) {
      std::lock_guard<std::mutex> lock(S->mu);
      S->fatal = err;
      for (auto &sl : S->active) {
        Out o;
        o.status = err;
        S->done[sl.req.ticket] = std::move(o);
      }
      S->active.clear();
      S->cv_done.notify_all();
      continue;
    }
    // retire finished structures; the survivors are repacked at the next admission or now
    std::vector<Slot> fin, keep;
    for (auto &sl : S->active) (sl.step >= sl.req.n_steps ? fin : keep).push_back(sl);
    if (!fin.empty()) {
      retire(S, fin);
      std::vector<Req> none;
      repack(S, keep, none, &err);
    }
  }
}

extern "C" fnn_status fnn_serve_create(fnn_server **out, fnn_ctx *ctx, size_t hbm_budget_bytes, fnn_precision prec,
                                       int32_t rebuild_every) {
  if (!out || !ctx || hbm_budget_bytes == 0 || rebuild_every < 1 ||
      (prec != FNN_FP32 && prec != FNN_BF16 && prec != FNN_FP32X3))
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
  fnn_status st = fnn_nlist_create(ctx, &S->nl, 0);
  if (st) {
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
  if (q->n_atoms * S->bytes_per_atom > (double)S->budget) return FNN_E_OOM;   // alone it exceeds the budget
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
  for (int b = 0; b < 2; b++) {
    if (S->Z[b]) cudaFree(S->Z[b]);
    if (S->pos[b]) cudaFree(S->pos[b]);
    if (S->vel[b]) cudaFree(S->vel[b]);
  }
  void *ptrs[] = {S->F, S->mol_offsets, S->mol_step, S->mol_nsteps, S->cell, S->pbc, S->E, S->hist_off,
                  S->hist_buf[0], S->hist_buf[1], S->mol_dt};
  for (void *p : ptrs)
    if (p) cudaFree(p);
  if (S->nl) fnn_nlist_destroy(S->nl);
  cudaStreamDestroy(S->stream);
  delete S;
  return FNN_OK;
}
