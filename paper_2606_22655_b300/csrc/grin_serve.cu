// grin_serve.cu -- continuous-batching trace server (grin_serve_* in grin.h).
//
// A scheduler thread owns all GPU work of a server.  Each round it
//   1. admits queued jobs, first come first served, while their device
//      footprint fits the free part of the arena (one cudaMalloc at
//      creation, carved by a first-fit allocator) and fewer than kMaxRunning
//      jobs run; admission copies the job's rays to its arena block and
//      clears its counters and resident ray slots;
//   2. launches one tick per running job on the job's own stream: every
//      resident slot advances its ray by up to step_quantum steps and takes
//      the job's next ray when one ends (k_serve_tick); the ticks of
//      different jobs run concurrently on the GPU;
//   3. waits for the ticks, reads each job's finished-ray counter, starts the
//      copy of the results of complete jobs to the caller's host buffers and
//      retires the jobs whose copy has ended.
// No device-side wait is involved: every tick is a bounded kernel (each slot
// runs at most step_quantum steps), so the GPU is never held by a spin.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "grin_internal.h"

namespace {

constexpr int kMaxRunning = 64;
constexpr size_t kAlign = 256;

size_t round_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

double now_s() {
  using namespace std::chrono;
  return duration<double>(steady_clock::now().time_since_epoch()).count();
}

// First-fit allocator over [0, capacity) with coalescing frees.
class Arena {
 public:
  explicit Arena(size_t cap) : cap_(cap) { free_[0] = cap; }
  bool alloc(size_t n, size_t* off) {
    n = round_up(n, kAlign);
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= n) {
        *off = it->first;
        size_t rest = it->second - n;
        size_t start = it->first + n;
        free_.erase(it);
        if (rest) free_[start] = rest;
        used_ += n;
        return true;
      }
    }
    return false;
  }
  void release(size_t off, size_t n) {
    n = round_up(n, kAlign);
    used_ -= n;
    auto it = free_.emplace(off, n).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_.erase(nx);
    }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_.erase(it);
      }
    }
  }
  size_t capacity() const { return cap_; }
  size_t used() const { return used_; }

 private:
  size_t cap_, used_ = 0;
  std::map<size_t, size_t> free_;
};

struct Job {
  uint64_t id = 0;
  grin_medium med = nullptr;
  grin_rays rays{};
  grin_params prm{};
  grin_out out{};
  int state = GRIN_JOB_QUEUED;  // written with the server lock held
  double t_submit = 0.0, t_admit = 0.0, t_done = 0.0;
  std::atomic<bool> cancel{false};  // set by grin_serve_cancel
  bool copying = false, failed = false;  // scheduler thread only
  // device resources while admitted
  size_t off = 0, bytes = 0;
  int nslots = 0;
  cudaStream_t stream = nullptr;
  cudaEvent_t ev = nullptr;
  unsigned long long* counters = nullptr;
  void* slots = nullptr;
  grin::TraceArgs args{};
  unsigned long long* host_done = nullptr;  // pinned
};

// Device layout of a job: counters | rays in | results | slot states |
// claim order (gridded media with enough rays; see ray_order.cu).
struct Layout {
  size_t counters, in, out, slots, order, total;
};

bool job_ordered(const grin::DevMedium& m, int64_t n) {
  return m.kind == GRIN_MEDIUM_GRID && n >= grin::kOrderMinRays && n < (int64_t(1) << 31);
}

Layout layout_of(int64_t n, int dtype, int nslots, bool ordered) {
  Layout L;
  const size_t esz = dtype == GRIN_F64 ? 8 : 4;
  L.counters = 0;
  L.in = kAlign;
  L.out = L.in + round_up(6 * esz * (size_t)n, kAlign);
  L.slots = L.out + round_up((7 * 8 + 4 * 4) * (size_t)n, kAlign);
  L.order = L.slots + round_up(grin::serve_slot_bytes() * (size_t)nslots, kAlign);
  L.total = L.order + (ordered ? round_up(grin::order_scratch_bytes(n), kAlign) : 0);
  return L;
}

}  // namespace

struct grin_server_s {
  grin_ctx ctx = nullptr;
  int quantum = 1024;
  int max_slots = 0;
  int slots_total = 0;
  unsigned char* arena_dev = nullptr;
  std::unique_ptr<Arena> arena;
  unsigned long long* pinned = nullptr;  // kMaxRunning finished-ray counters
  std::vector<int> pinned_free;
  std::mutex mu;
  std::condition_variable cv;
  std::map<uint64_t, std::shared_ptr<Job>> jobs;
  std::deque<std::shared_ptr<Job>> queue;
  std::vector<std::shared_ptr<Job>> running;
  uint64_t next_id = 1;
  bool stop = false;
  std::thread thread;
  grin_serve_counters st{};
};

namespace {

int job_slots(grin_server s, int64_t n) {
  int64_t want = (int64_t)round_up((size_t)n, 128);
  return (int)std::min<int64_t>(want, s->max_slots);
}

void retire(grin_server s, Job& j, int state) {
  if (j.stream) {
    cudaStreamSynchronize(j.stream);
    cudaStreamDestroy(j.stream);
    j.stream = nullptr;
  }
  if (j.ev) {
    cudaEventDestroy(j.ev);
    j.ev = nullptr;
  }
  if (j.bytes) {
    s->arena->release(j.off, j.bytes);
    j.bytes = 0;
  }
  if (j.host_done) {
    s->pinned_free.push_back((int)(j.host_done - s->pinned));
    j.host_done = nullptr;
  }
  j.state = state;
  j.t_done = now_s();
  if (state == GRIN_JOB_DONE) ++s->st.done;
  else if (state == GRIN_JOB_FAILED) ++s->st.failed;
  else if (state == GRIN_JOB_CANCELLED) ++s->st.cancelled;
}

// Admit queued jobs that fit (called with the lock held).
void admit(grin_server s) {
  while (!s->queue.empty() && (int)s->running.size() < kMaxRunning && !s->pinned_free.empty()) {
    std::shared_ptr<Job> jp = s->queue.front();
    Job& j = *jp;
    if (j.cancel) {
      s->queue.pop_front();
      retire(s, j, GRIN_JOB_CANCELLED);
      continue;
    }
    const int64_t n = j.rays.count;
    j.nslots = job_slots(s, n);
    const bool ordered = job_ordered(j.med->dm, n);
    Layout L = layout_of(n, j.rays.dtype, j.nslots, ordered);
    size_t off;
    if (!s->arena->alloc(L.total, &off)) break;  // first come first served: wait
    s->queue.pop_front();
    j.t_admit = now_s();
    j.off = off;
    j.bytes = L.total;
    j.host_done = s->pinned + s->pinned_free.back();
    s->pinned_free.pop_back();
    *j.host_done = 0;
    unsigned char* base = s->arena_dev + off;
    j.counters = (unsigned long long*)(base + L.counters);
    j.slots = base + L.slots;
    const size_t esz = j.rays.dtype == GRIN_F64 ? 8 : 4;
    bool ok = cudaStreamCreateWithFlags(&j.stream, cudaStreamNonBlocking) == cudaSuccess &&
              cudaEventCreateWithFlags(&j.ev, cudaEventDisableTiming) == cudaSuccess;
    const void* hin[6] = {j.rays.ox, j.rays.oy, j.rays.oz, j.rays.dx, j.rays.dy, j.rays.dz};
    void* din[6];
    for (int k = 0; k < 6 && ok; ++k) {
      din[k] = base + L.in + (size_t)k * esz * (size_t)n;
      ok = cudaMemcpyAsync(din[k], hin[k], esz * (size_t)n, cudaMemcpyHostToDevice, j.stream) ==
           cudaSuccess;
    }
    ok = ok && cudaMemsetAsync(j.counters, 0, 2 * sizeof(unsigned long long), j.stream) == cudaSuccess;
    ok = ok && cudaMemsetAsync(j.slots, 0, grin::serve_slot_bytes() * (size_t)j.nslots, j.stream) ==
                   cudaSuccess;
    if (!ok) {
      cudaGetLastError();
      retire(s, j, GRIN_JOB_FAILED);
      continue;
    }
    unsigned char* ob = base + L.out;
    grin::TraceArgs& a = j.args;
    a.ox = din[0];
    a.oy = din[1];
    a.oz = din[2];
    a.dx = din[3];
    a.dy = din[4];
    a.dz = din[5];
    a.count = n;
    a.dtype = j.rays.dtype;
    double* dd[7];
    for (int k = 0; k < 7; ++k) dd[k] = (double*)(ob + (size_t)k * 8 * (size_t)n);
    int32_t* di[4];
    for (int k = 0; k < 4; ++k) di[k] = (int32_t*)(ob + 56 * (size_t)n + (size_t)k * 4 * (size_t)n);
    a.px = dd[0];
    a.py = dd[1];
    a.pz = dd[2];
    a.ux = dd[3];
    a.uy = dd[4];
    a.uz = dd[5];
    a.opl = dd[6];
    a.exit_id = di[0];
    a.steps = di[1];
    a.tir_i = di[2];
    a.tir_b = di[3];
    a.dopl = j.prm.dopl;
    a.max_steps = j.prm.max_steps;
    a.flags = j.prm.flags;
    a.perm = nullptr;
    // gridded media: claim the job's rays in entry-cell order (ray_order.cu)
    if (ordered && grin::launch_order(j.med->dm, a, base + L.order, s->ctx->sm_count, j.stream,
                                      &a.perm) < 0) {
      cudaGetLastError();
      a.perm = nullptr;
    }
    j.state = GRIN_JOB_RUNNING;
    s->running.push_back(jp);
  }
}

void start_copy_out(Job& j) {
  const grin::TraceArgs& a = j.args;
  const size_t n = (size_t)a.count;
  double* hd[7] = {j.out.px, j.out.py, j.out.pz, j.out.dx, j.out.dy, j.out.dz, j.out.opl};
  const double* dd[7] = {a.px, a.py, a.pz, a.ux, a.uy, a.uz, a.opl};
  int32_t* hi[4] = {j.out.exit_id, j.out.steps, j.out.tir_internal, j.out.tir_boundary};
  const int32_t* di[4] = {a.exit_id, a.steps, a.tir_i, a.tir_b};
  for (int k = 0; k < 7; ++k) cudaMemcpyAsync(hd[k], dd[k], 8 * n, cudaMemcpyDeviceToHost, j.stream);
  for (int k = 0; k < 4; ++k) cudaMemcpyAsync(hi[k], di[k], 4 * n, cudaMemcpyDeviceToHost, j.stream);
  cudaEventRecord(j.ev, j.stream);
  j.copying = true;
}

void scheduler(grin_server s) {
  cudaSetDevice(s->ctx->device);
  std::unique_lock<std::mutex> lock(s->mu);
  while (!s->stop) {
    admit(s);
    if (s->running.empty()) {
      s->cv.wait_for(lock, std::chrono::milliseconds(50));
      continue;
    }
    std::vector<std::shared_ptr<Job>> run = s->running;
    lock.unlock();
    // ticks
    int ticked = 0;
    for (auto& jp : run) {
      Job& j = *jp;
      if (j.copying || j.cancel || j.failed) continue;
      ++ticked;
      int rc = grin::launch_serve_tick(j.med->dm, j.args, j.slots, j.nslots, j.counters, s->quantum,
                                       j.stream);
      if (rc < 0) {
        cudaGetLastError();
        j.failed = true;
        continue;
      }
      cudaMemcpyAsync(j.host_done, j.counters + 1, sizeof(unsigned long long),
                      cudaMemcpyDeviceToHost, j.stream);
    }
    for (auto& jp : run) {
      Job& j = *jp;
      if (j.copying || j.cancel || j.failed) continue;
      if (cudaStreamSynchronize(j.stream) != cudaSuccess) {
        cudaGetLastError();
        j.failed = true;
        continue;
      }
      if (*j.host_done >= (unsigned long long)j.args.count) start_copy_out(j);
    }
    lock.lock();
    ++s->st.ticks;
    // retire finished, failed and cancelled jobs
    std::vector<std::shared_ptr<Job>> keep;
    for (auto& jp : s->running) {
      Job& j = *jp;
      if (j.failed) {
        retire(s, j, GRIN_JOB_FAILED);
      } else if (j.cancel) {
        retire(s, j, GRIN_JOB_CANCELLED);
      } else if (j.copying && cudaEventQuery(j.ev) == cudaSuccess) {
        double steps = 0.0;
        for (int64_t i = 0; i < j.args.count; ++i) steps += (double)j.out.steps[i];
        s->st.ray_steps += steps;
        retire(s, j, GRIN_JOB_DONE);
      } else {
        keep.push_back(jp);
      }
    }
    if (keep.size() != s->running.size()) s->cv.notify_all();
    s->running.swap(keep);
    // every running job is copying its results out: wait a little (a new
    // submission wakes the loop) instead of polling the copies at once
    if (!ticked && !s->running.empty() && s->queue.empty())
      s->cv.wait_for(lock, std::chrono::microseconds(200));
  }
  // shutdown: everything still here is cancelled
  for (auto& jp : s->running) retire(s, *jp, GRIN_JOB_CANCELLED);
  s->running.clear();
  for (auto& jp : s->queue) retire(s, *jp, GRIN_JOB_CANCELLED);
  s->queue.clear();
  s->cv.notify_all();
}

bool finished(int state) {
  return state == GRIN_JOB_DONE || state == GRIN_JOB_FAILED || state == GRIN_JOB_CANCELLED;
}

}  // namespace

extern "C" {

int grin_serve_create(grin_ctx ctx, const grin_serve_config* cfg, grin_server* out) {
  if (!ctx || !cfg || !out || cfg->hbm_budget_bytes == 0 || cfg->step_quantum < 0 ||
      cfg->max_slots_per_job < 0)
    return GRIN_ERR_INVALID_ARG;
  *out = nullptr;
  grin_server s = new (std::nothrow) grin_server_s;
  if (!s) return GRIN_ERR_OOM;
  s->ctx = ctx;
  s->quantum = cfg->step_quantum > 0 ? cfg->step_quantum : 1024;
  // one tick kernel fills the GPU with 5 blocks of 128 threads per SM
  s->slots_total = ctx->sm_count * 5 * 128;
  int cap = cfg->max_slots_per_job > 0 ? cfg->max_slots_per_job : s->slots_total;
  s->max_slots = std::max(128, (int)round_up((size_t)cap, 128));
  cudaSetDevice(ctx->device);
  if (cudaMalloc(&s->arena_dev, cfg->hbm_budget_bytes) != cudaSuccess) {
    cudaGetLastError();
    delete s;
    return GRIN_ERR_OOM;
  }
  if (cudaHostAlloc(&s->pinned, kMaxRunning * sizeof(unsigned long long), cudaHostAllocDefault) !=
      cudaSuccess) {
    cudaGetLastError();
    cudaFree(s->arena_dev);
    delete s;
    return GRIN_ERR_OOM;
  }
  for (int k = kMaxRunning - 1; k >= 0; --k) s->pinned_free.push_back(k);
  s->arena.reset(new Arena(cfg->hbm_budget_bytes));
  s->st.arena_bytes = cfg->hbm_budget_bytes;
  s->st.slots_total = s->slots_total;
  s->thread = std::thread(scheduler, s);
  ++ctx->children;
  *out = s;
  return GRIN_OK;
}

int grin_serve_destroy(grin_server s) {
  if (!s) return GRIN_ERR_INVALID_ARG;
  {
    std::lock_guard<std::mutex> lock(s->mu);
    s->stop = true;
  }
  s->cv.notify_all();
  if (s->thread.joinable()) s->thread.join();
  cudaSetDevice(s->ctx->device);
  cudaFree(s->arena_dev);
  cudaFreeHost(s->pinned);
  --s->ctx->children;
  delete s;
  return GRIN_OK;
}

int grin_serve_submit(grin_server s, grin_medium med, const grin_rays* rays, const grin_params* p,
                      const grin_out* out, uint64_t* job_id) {
  if (!s || !med || !rays || !p || !out || !job_id) return GRIN_ERR_INVALID_ARG;
  if (med->ctx != s->ctx || rays->count < 0) return GRIN_ERR_INVALID_ARG;
  if (rays->dtype != GRIN_F32 && rays->dtype != GRIN_F64) return GRIN_ERR_INVALID_ARG;
  if (p->precision != GRIN_PREC_FP32_MIXED || !(p->dopl > 0.0) || p->max_steps < 0 ||
      (p->flags & ~(uint32_t)GRIN_TRACE_LEVEL_ROOT))
    return GRIN_ERR_INVALID_ARG;
  if (out->margin) return GRIN_ERR_NOT_IMPLEMENTED;
  if (rays->count > 0) {
    if (!rays->ox || !rays->oy || !rays->oz || !rays->dx || !rays->dy || !rays->dz)
      return GRIN_ERR_INVALID_ARG;
    if (!out->px || !out->py || !out->pz || !out->dx || !out->dy || !out->dz || !out->opl ||
        !out->exit_id || !out->steps || !out->tir_internal || !out->tir_boundary)
      return GRIN_ERR_INVALID_ARG;
    Layout L = layout_of(rays->count, rays->dtype, job_slots(s, rays->count),
                         job_ordered(med->dm, rays->count));
    if (round_up(L.total, kAlign) > s->arena->capacity()) return GRIN_ERR_BUSY;
  }
  auto j = std::make_shared<Job>();
  j->med = med;
  j->rays = *rays;
  j->prm = *p;
  j->out = *out;
  j->t_submit = now_s();
  std::lock_guard<std::mutex> lock(s->mu);
  if (s->stop) return GRIN_ERR_CANCELLED;
  j->id = s->next_id++;
  s->jobs[j->id] = j;
  ++s->st.submitted;
  if (rays->count == 0) {
    j->state = GRIN_JOB_DONE;
    j->t_done = now_s();
    ++s->st.done;
  } else {
    s->queue.push_back(j);
  }
  *job_id = j->id;
  s->cv.notify_all();
  return GRIN_OK;
}

int grin_serve_timing(grin_server s, uint64_t id, double* queued_s, double* run_s) {
  if (!s || !queued_s || !run_s) return GRIN_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lock(s->mu);
  auto it = s->jobs.find(id);
  if (it == s->jobs.end()) return GRIN_ERR_NOT_FOUND;
  const Job& j = *it->second;
  const double now = now_s();
  const bool admitted = j.t_admit > 0.0;
  const double end = finished(j.state) ? j.t_done : now;
  *queued_s = (admitted ? j.t_admit : end) - j.t_submit;
  *run_s = admitted ? end - j.t_admit : 0.0;
  return GRIN_OK;
}

int grin_serve_poll(grin_server s, uint64_t id, int32_t* state, double* latency_s) {
  if (!s || !state) return GRIN_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lock(s->mu);
  auto it = s->jobs.find(id);
  if (it == s->jobs.end()) return GRIN_ERR_NOT_FOUND;
  Job& j = *it->second;
  *state = j.state;
  if (latency_s) *latency_s = (finished(j.state) ? j.t_done : now_s()) - j.t_submit;
  return GRIN_OK;
}

int grin_serve_wait(grin_server s, uint64_t id, double timeout_s, int32_t* state) {
  if (!s) return GRIN_ERR_INVALID_ARG;
  std::unique_lock<std::mutex> lock(s->mu);
  auto it = s->jobs.find(id);
  if (it == s->jobs.end()) return GRIN_ERR_NOT_FOUND;
  std::shared_ptr<Job> jp = it->second;
  bool ok = s->cv.wait_for(lock, std::chrono::duration<double>(std::max(0.0, timeout_s)),
                           [&] { return finished(jp->state); });
  if (state) *state = jp->state;
  return ok ? GRIN_OK : GRIN_ERR_TIMEOUT;
}

int grin_serve_cancel(grin_server s, uint64_t id) {
  if (!s) return GRIN_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lock(s->mu);
  auto it = s->jobs.find(id);
  if (it == s->jobs.end()) return GRIN_ERR_NOT_FOUND;
  Job& j = *it->second;
  if (finished(j.state)) return GRIN_OK;
  j.cancel = true;
  if (j.state == GRIN_JOB_QUEUED) {
    auto q = std::find(s->queue.begin(), s->queue.end(), it->second);
    if (q != s->queue.end()) s->queue.erase(q);
    retire(s, j, GRIN_JOB_CANCELLED);
    s->cv.notify_all();
  }
  return GRIN_OK;
}

int grin_serve_stats(grin_server s, grin_serve_counters* out) {
  if (!s || !out) return GRIN_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lock(s->mu);
  *out = s->st;
  out->arena_in_use = s->arena->used();
  int slots = 0;
  for (auto& j : s->running) slots += j->nslots;
  out->slots_in_use = slots;
  out->jobs_queued = (int)s->queue.size();
  out->jobs_running = (int)s->running.size();
  return GRIN_OK;
}

}  // extern "C"
