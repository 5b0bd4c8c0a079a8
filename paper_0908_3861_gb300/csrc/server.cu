// Serving: a request loop for filter jobs on one GPU (host code).
//
// One worker thread owns the device work.  Submitted jobs wait in a FIFO
// queue.  The worker admits a job when a slot (one of max_inflight CUDA
// streams) is free and the job's device footprint fits the HBM budget --
// evicting least-recently-used resident integrated images if that makes room
// -- and later jobs that fit may pass a head job that does not.  An admitted
// job allocates its buffers stream-ordered (cudaMallocAsync), copies its
// inputs in, runs abf_integrate and abf_filter on its stream, copies the
// output out and records an event; jobs on different streams overlap on the
// device.  The worker polls the events, frees finished jobs' buffers (or keeps
// the integrated image resident under its image id) and wakes waiters.
// Every wait is bounded: abf_wait takes a timeout and returns
// ABF_ERR_TIMEOUT when it runs out.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <list>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "abf_internal.cuh"

namespace {

double now_us() {
  using namespace std::chrono;
  return (double)duration_cast<nanoseconds>(steady_clock::now().time_since_epoch()).count() * 1e-3;
}

size_t elem_bytes(int dtype) { return dtype == ABF_U8 ? 1 : dtype == ABF_U16 ? 2 : dtype == ABF_F32 ? 4 : 8; }

struct Resident {
  uint64_t image_id;
  std::string key;  // descriptor bytes
  void* d_g;
  size_t bytes;
  int users;        // running jobs reading it
  double last_use;
};

struct Job {
  uint64_t ticket;
  abf_request req;
  abf_plan plan = nullptr;
  std::string key;
  void *d_f = nullptr, *d_sc = nullptr, *d_s = nullptr, *d_g = nullptr, *d_ws = nullptr;
  size_t bytes = 0;        // footprint charged to the budget
  int slot = -1;
  cudaEvent_t ev = nullptr;     // end of the job's stream work (timed)
  cudaEvent_t ev0 = nullptr;    // start of the job's stream work (timed)
  cudaEvent_t ev_ready = nullptr;  // grouped jobs: integrated image and scales on the device
  Resident* res = nullptr; // integrated image reused from / kept in the resident set
  Resident* pinned = nullptr;  // resident image held since submit (a request without h_f)
  bool keep = false;       // keep d_g resident after the job
  abf_job_stats st{};
  int state = 0;           // 0 queued, 1 running, 2 done
};

}  // namespace

struct abf_server_s {
  abf_server_cfg cfg{};
  int device = 0;
  std::thread worker;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Job*> queue;
  std::vector<Job*> running;
  std::unordered_map<uint64_t, Job*> jobs;
  std::list<Resident> resident;
  std::map<std::string, abf_plan> plans;
  std::vector<cudaStream_t> streams;
  std::vector<int> slot_busy;
  int32_t* h_dev_status = nullptr;  // pinned, one word per slot
  int32_t* d_slot_status = nullptr; // device status word per slot, cleared before every job
  unsigned long long* d_slot_counter = nullptr;  // 32 work counters per slot (grouped mesh launches)
  cudaEvent_t base_ev = nullptr;    // device-clock origin of the job timestamps
  size_t used = 0, peak = 0;
  uint64_t next_ticket = 1;
  bool stop = false, paused = false;

  static std::string key_of(const abf_desc& d) { return std::string((const char*)&d, sizeof(d)); }

  abf_plan plan_for(const abf_desc& d, abf_status* s) {
    const std::string k = key_of(d);
    auto it = plans.find(k);
    if (it != plans.end()) {
      *s = ABF_OK;
      return it->second;
    }
    abf_plan p = nullptr;
    *s = abf_plan_create(&d, &p);
    if (*s == ABF_OK) plans[k] = p;
    return p;
  }

  Resident* find_resident(uint64_t id, const std::string& key) {
    if (!id) return nullptr;
    for (auto& r : resident)
      if (r.image_id == id && r.key == key) return &r;
    return nullptr;
  }

  // Free resident images (least recently used first, not in use) until
  // `need` more bytes fit the budget.  Returns whether they fit.
  bool make_room(size_t need, cudaStream_t st) {
    while (used + need > cfg.hbm_budget) {
      auto victim = resident.end();
      for (auto it = resident.begin(); it != resident.end(); ++it)
        if (it->users == 0 && (victim == resident.end() || it->last_use < victim->last_use)) victim = it;
      if (victim == resident.end()) return false;
      cudaFreeAsync(victim->d_g, st);
      used -= victim->bytes;
      resident.erase(victim);
    }
    return true;
  }

  void finish(Job* j, abf_status s) {
    j->st.status = s;
    j->st.t_done_us = now_us();
    j->state = 2;
    cv_done.notify_all();
  }

  // Start a job on a free slot; false if it cannot start now (no room).  With
  // `defer`, the job stops after its non-adaptive step (ev_ready recorded) and
  // its adaptive step runs in a grouped launch (launch_group); otherwise it
  // runs to the end on its own stream.  *started tells whether it is now
  // running (a job that failed at once is finished instead).
  bool try_start(Job* j, int slot, bool defer, bool* started) {
    *started = false;
    cudaStream_t st = streams[slot];
    abf_status s;
    j->plan = plan_for(j->req.desc, &s);
    if (s != ABF_OK) {
      unpin(j);
      finish(j, s);
      return true;
    }
    if (defer && !grouping_ok(j->plan)) defer = false;
    const abf_plan p = j->plan;
    const int W = p->pv.W, H = p->pv.H;
    const size_t fb = (size_t)W * H * elem_bytes(p->pv.in_dtype), sb = (size_t)W * H * 16,
                 ob = (size_t)W * H * elem_bytes(p->pv.out_dtype);
    // a request without an image uses the resident image held since submit
    j->res = j->pinned ? j->pinned : find_resident(j->req.image_id, j->key);
    const bool hit = j->res != nullptr;
    const size_t need = (hit ? 0 : fb + p->g_bytes + p->ws_bytes) + sb + ob;
    if (!make_room(need, st)) return false;
    j->bytes = need;
    used += need;
    peak = std::max(peak, used);
    j->slot = slot;
    slot_busy[slot] = 1;
    j->st.t_admit_us = now_us();
    j->state = 1;
    running.push_back(j);
    cudaError_t e = cudaSuccess;
    auto ok = [&](cudaError_t r) { if (e == cudaSuccess) e = r; };
    int32_t* dst = d_slot_status + slot;
    ok(cudaEventCreate(&j->ev0));
    if (e == cudaSuccess) ok(cudaEventRecord(j->ev0, st));
    ok(cudaMemsetAsync(dst, 0, sizeof(int32_t), st));
    ok(abf::fault_take(ABF_FAULT_ALLOC) ? cudaErrorMemoryAllocation : cudaMallocAsync(&j->d_sc, sb, st));
    ok(cudaMallocAsync(&j->d_s, ob, st));
    if (e == cudaSuccess)
      ok(cudaMemcpy2DAsync(j->d_sc, (size_t)W * 16, j->req.h_scales, j->req.scale_pitch, (size_t)W * 16, H,
                           cudaMemcpyHostToDevice, st));
    if (hit) {
      j->d_g = j->res->d_g;
      if (!j->pinned) j->res->users++;  // a pinned image was counted at submit
      j->pinned = nullptr;              // from here on released through j->res
      j->res->last_use = now_us();
      j->st.resident_hit = 1;
    } else {
      ok(cudaMallocAsync(&j->d_f, fb, st));
      ok(cudaMallocAsync(&j->d_g, p->g_bytes, st));
      ok(cudaMallocAsync(&j->d_ws, p->ws_bytes, st));
      if (e == cudaSuccess)
        ok(cudaMemcpy2DAsync(j->d_f, (size_t)W * elem_bytes(p->pv.in_dtype), j->req.h_f, j->req.f_pitch,
                             (size_t)W * elem_bytes(p->pv.in_dtype), H, cudaMemcpyHostToDevice, st));
      if (e == cudaSuccess && abf::integrate_with_status(p, j->d_f, (size_t)W * elem_bytes(p->pv.in_dtype), j->d_g,
                                                         j->d_ws, dst, st) != ABF_OK)
        e = cudaErrorLaunchFailure;
    }
    if (defer) {
      if (e == cudaSuccess) ok(cudaEventCreateWithFlags(&j->ev_ready, cudaEventDisableTiming));
      if (e == cudaSuccess) ok(cudaEventRecord(j->ev_ready, st));
      if (e != cudaSuccess) {
        cudaGetLastError();
        complete(j, e == cudaErrorMemoryAllocation ? ABF_ERR_OOM : ABF_ERR_CUDA);
        return true;
      }
      *started = true;
      return true;
    }
    if (e == cudaSuccess &&
        abf::filter_with_status(p, j->d_g, j->d_sc, (size_t)W * 16, j->d_s, (size_t)W * elem_bytes(p->pv.out_dtype),
                                dst, st) != ABF_OK)
      e = cudaErrorLaunchFailure;
    finish_tail(j, e);
    return true;
  }

  // The end of a job's stream work: output and status word back to the host,
  // the end event; or the job's completion with an error.
  void finish_tail(Job* j, cudaError_t e) {
    cudaStream_t st = streams[j->slot];
    const abf_plan p = j->plan;
    const int W = p->pv.W, H = p->pv.H;
    auto ok = [&](cudaError_t r) { if (e == cudaSuccess) e = r; };
    if (e == cudaSuccess)
      ok(cudaMemcpy2DAsync(j->req.h_s, j->req.s_pitch, j->d_s, (size_t)W * elem_bytes(p->pv.out_dtype),
                           (size_t)W * elem_bytes(p->pv.out_dtype), H, cudaMemcpyDeviceToHost, st));
    if (e == cudaSuccess)
      ok(cudaMemcpyAsync(&h_dev_status[j->slot], d_slot_status + j->slot, sizeof(int32_t), cudaMemcpyDeviceToHost,
                         st));
    if (e == cudaSuccess) ok(cudaEventCreate(&j->ev));
    if (e == cudaSuccess) ok(cudaEventRecord(j->ev, st));
    if (e != cudaSuccess) {
      cudaGetLastError();
      complete(j, e == cudaErrorMemoryAllocation ? ABF_ERR_OOM : ABF_ERR_CUDA);
    }
  }

  // Jobs whose adaptive step may share a grouped launch: exact-form plans of
  // the four-direction filter with phi = delta (the batched mesh runs every
  // order and limb count of those).
  static bool grouping_ok(abf_plan p) { return p && p->desc.form == ABF_FORM_EXACT && !p->general; }

  // The adaptive step of jobs admitted together, in one batched launch per
  // (order, limbs) group on the first job's stream, after every job's own
  // non-adaptive step; each job's stream then copies its result out.
  void launch_group(std::vector<Job*>& grp) {
    if (grp.empty()) return;
    if (grp.size() == 1) {
      Job* j = grp[0];
      cudaError_t e = cudaStreamWaitEvent(streams[j->slot], j->ev_ready, 0);
      const abf_plan p = j->plan;
      const int W = p->pv.W;
      if (e == cudaSuccess &&
          abf::filter_with_status(p, j->d_g, j->d_sc, (size_t)W * 16, j->d_s,
                                  (size_t)W * elem_bytes(p->pv.out_dtype), d_slot_status + j->slot,
                                  streams[j->slot]) != ABF_OK)
        e = cudaErrorLaunchFailure;
      finish_tail(j, e);
      return;
    }
    cudaStream_t gs = streams[grp[0]->slot];
    cudaError_t e = cudaSuccess;
    std::vector<abf::BatchIn> in;
    for (Job* j : grp) {
      if (e == cudaSuccess) e = cudaStreamWaitEvent(gs, j->ev_ready, 0);
      const abf_plan p = j->plan;
      const int W = p->pv.W;
      in.push_back(abf::BatchIn{p->pv, (const uint64_t*)j->d_g, j->d_sc, (size_t)W * 16, j->d_s,
                                (size_t)W * elem_bytes(p->pv.out_dtype), d_slot_status + j->slot});
    }
    if (e == cudaSuccess) e = abf::run_mesh_batch(in.data(), (int)in.size(), d_slot_counter + 32 * grp[0]->slot, 8, gs);
    cudaEvent_t meshed = nullptr;
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&meshed, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventRecord(meshed, gs);
    for (Job* j : grp) {
      cudaError_t ej = e;
      if (ej == cudaSuccess) ej = cudaStreamWaitEvent(streams[j->slot], meshed, 0);
      finish_tail(j, ej);
    }
    if (meshed) cudaEventDestroy(meshed);
  }

  // Release the resident image a request without h_f has held since submit.
  void unpin(Job* j) {
    if (j->pinned) {
      j->pinned->users--;
      j->pinned = nullptr;
    }
  }

  // Release a running job's resources (after its event completed, or on error).
  void complete(Job* j, abf_status s) {
    cudaStream_t st = streams[j->slot];
    if (j->ev) {
      j->st.device_status = h_dev_status[j->slot];
      float a = 0.f, b = 0.f;
      if (s == ABF_OK && cudaEventElapsedTime(&a, base_ev, j->ev0) == cudaSuccess &&
          cudaEventElapsedTime(&b, base_ev, j->ev) == cudaSuccess) {
        j->st.t_gpu_start_us = 1e3 * (double)a;
        j->st.t_gpu_end_us = 1e3 * (double)b;
      }
      cudaGetLastError();
      cudaEventDestroy(j->ev);
      j->ev = nullptr;
    }
    if (j->ev0) {
      cudaEventDestroy(j->ev0);
      j->ev0 = nullptr;
    }
    if (j->ev_ready) {
      cudaEventDestroy(j->ev_ready);
      j->ev_ready = nullptr;
    }
    size_t freed = 0;
    const abf_plan p = j->plan;
    const int W = p->pv.W, H = p->pv.H;
    if (j->d_sc) cudaFreeAsync(j->d_sc, st);
    if (j->d_s) cudaFreeAsync(j->d_s, st);
    freed += (size_t)W * H * 16 + (size_t)W * H * elem_bytes(p->pv.out_dtype);
    if (j->res) {
      j->res->users--;
    } else {
      if (j->d_f) cudaFreeAsync(j->d_f, st);
      if (j->d_ws) cudaFreeAsync(j->d_ws, st);
      freed += (size_t)W * H * elem_bytes(p->pv.in_dtype) + p->ws_bytes;
      if (j->req.image_id && s == ABF_OK) {
        resident.push_back(Resident{j->req.image_id, j->key, j->d_g, p->g_bytes, 0, now_us()});
      } else {
        if (j->d_g) cudaFreeAsync(j->d_g, st);
        freed += p->g_bytes;
      }
    }
    used -= std::min(used, freed);
    slot_busy[j->slot] = 0;
    running.erase(std::remove(running.begin(), running.end(), j), running.end());
    finish(j, s);
  }

  void loop() {
    cudaSetDevice(device);
    std::unique_lock<std::mutex> lk(mu);
    for (;;) {
      bool progress = false;
      // completions
      for (size_t i = 0; i < running.size();) {
        Job* j = running[i];
        const cudaError_t q = cudaEventQuery(j->ev);
        if (q == cudaErrorNotReady) {
          ++i;
          continue;
        }
        if (q != cudaSuccess) cudaGetLastError();
        complete(j, q == cudaSuccess ? ABF_OK : ABF_ERR_CUDA);
        progress = true;
      }
      // admissions, in arrival order; a job that does not fit lets later ones
      // try.  With grouping on, the jobs admitted in one round share one
      // batched launch of the adaptive step.
      if (!paused && !abf::fault_active(ABF_FAULT_QUEUE_STALL)) {
        const bool grouping = (cfg.flags & ABF_SERVER_GROUP_MESH) != 0;
        std::vector<Job*> grp;
        for (auto it = queue.begin(); it != queue.end();) {
          int slot = -1;
          for (int k = 0; k < (int)slot_busy.size(); ++k)
            if (!slot_busy[k]) { slot = k; break; }
          if (slot < 0) break;
          Job* j = *it;
          bool started = false;
          if (try_start(j, slot, grouping, &started)) {
            it = queue.erase(it);
            progress = true;
            if (started) grp.push_back(j);
          } else {
            ++it;
          }
        }
        launch_group(grp);
      }
      if (stop && queue.empty() && running.empty()) break;
      if (!progress) cv_work.wait_for(lk, std::chrono::microseconds(running.empty() ? 2000 : 50));
    }
  }
};

extern "C" {

abf_status abf_server_create(const abf_server_cfg* cfg, abf_server* out) {
  if (!cfg || !out || cfg->hbm_budget == 0 || cfg->max_inflight < 1 || cfg->max_inflight > 64) return ABF_ERR_INVALID;
  if (cfg->flags & ~ABF_SERVER_GROUP_MESH) return ABF_ERR_INVALID;
  *out = nullptr;
  abf_server s = new (std::nothrow) abf_server_s();
  if (!s) return ABF_ERR_OOM;
  s->cfg = *cfg;
  if (cudaGetDevice(&s->device) != cudaSuccess) { delete s; return ABF_ERR_CUDA; }
  s->streams.resize(cfg->max_inflight);
  s->slot_busy.assign(cfg->max_inflight, 0);
  for (auto& st : s->streams)
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) { delete s; return ABF_ERR_CUDA; }
  if (cudaHostAlloc((void**)&s->h_dev_status, sizeof(int32_t) * cfg->max_inflight, cudaHostAllocDefault) != cudaSuccess) {
    delete s;
    return ABF_ERR_CUDA;
  }
  if (cudaMalloc((void**)&s->d_slot_status, sizeof(int32_t) * cfg->max_inflight) != cudaSuccess) {
    cudaFreeHost(s->h_dev_status);
    delete s;
    return ABF_ERR_CUDA;
  }
  if (cudaMalloc((void**)&s->d_slot_counter, sizeof(unsigned long long) * 32 * cfg->max_inflight) != cudaSuccess) {
    cudaFreeHost(s->h_dev_status);
    cudaFree(s->d_slot_status);
    delete s;
    return ABF_ERR_CUDA;
  }
  if (cudaEventCreate(&s->base_ev) != cudaSuccess || cudaEventRecord(s->base_ev, s->streams[0]) != cudaSuccess ||
      cudaEventSynchronize(s->base_ev) != cudaSuccess) {
    cudaFreeHost(s->h_dev_status);
    cudaFree(s->d_slot_status);
    cudaFree(s->d_slot_counter);
    delete s;
    return ABF_ERR_CUDA;
  }
  s->worker = std::thread([s] { s->loop(); });
  *out = s;
  return ABF_OK;
}

abf_status abf_submit(abf_server s, const abf_request* req, uint64_t* ticket) {
  if (!s || !req || !ticket || !req->h_scales || !req->h_s) return ABF_ERR_INVALID;
  if (req->desc.form != ABF_FORM_EXACT) return ABF_ERR_UNSUPPORTED;
  const abf_desc& d = req->desc;
  if (d.width < 1 || d.height < 1) return ABF_ERR_INVALID;
  Job* j = new (std::nothrow) Job();
  if (!j) return ABF_ERR_OOM;
  j->req = *req;
  j->key = abf_server_s::key_of(d);
  j->st.t_submit_us = now_us();
  {
    std::lock_guard<std::mutex> lk(s->mu);
    abf_status ps;
    const abf_plan p = s->plan_for(d, &ps);
    if (ps != ABF_OK) {
      delete j;
      return ps;
    }
    // the whole footprint must fit the budget on its own, or it never runs
    const size_t px = (size_t)d.width * d.height;
    const size_t full = px * (16 + elem_bytes(d.out_dtype) + elem_bytes(d.in_dtype)) + p->g_bytes + p->ws_bytes;
    if (full > s->cfg.hbm_budget) {
      delete j;
      return ABF_ERR_BUSY;
    }
    if (!req->h_f) {
      // hold the resident image from now on, so that no eviction can take it
      // away before the job is admitted
      Resident* r = s->find_resident(req->image_id, j->key);
      if (!r) {
        delete j;
        return ABF_ERR_INVALID;
      }
      r->users++;
      j->pinned = r;
    }
    j->ticket = s->next_ticket++;
    s->jobs[j->ticket] = j;
    s->queue.push_back(j);
    *ticket = j->ticket;
  }
  s->cv_work.notify_one();
  return ABF_OK;
}

abf_status abf_poll(abf_server s, uint64_t ticket, int32_t* done, abf_job_stats* stats) {
  if (!s || !done) return ABF_ERR_INVALID;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->jobs.find(ticket);
  if (it == s->jobs.end()) return ABF_ERR_INVALID;
  *done = it->second->state == 2;
  if (*done && stats) *stats = it->second->st;
  return ABF_OK;
}

abf_status abf_wait(abf_server s, uint64_t ticket, int64_t timeout_us, abf_job_stats* stats) {
  if (!s) return ABF_ERR_INVALID;
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->jobs.find(ticket);
  if (it == s->jobs.end()) return ABF_ERR_INVALID;
  Job* j = it->second;
  auto pred = [&] { return j->state == 2; };
  if (timeout_us < 0) {
    s->cv_done.wait(lk, pred);
  } else if (!s->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us), pred)) {
    return ABF_ERR_TIMEOUT;
  }
  if (stats) *stats = j->st;
  const abf_status r = (abf_status)j->st.status;
  s->jobs.erase(it);
  delete j;
  return r;
}

abf_status abf_server_pause(abf_server s, int32_t paused) {
  if (!s) return ABF_ERR_INVALID;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->paused = paused != 0;
  }
  s->cv_work.notify_one();
  return ABF_OK;
}

abf_status abf_server_stats(abf_server s, size_t* used, size_t* peak, int32_t* inflight, int32_t* queued,
                            int32_t* resident) {
  if (!s) return ABF_ERR_INVALID;
  std::lock_guard<std::mutex> lk(s->mu);
  if (used) *used = s->used;
  if (peak) *peak = s->peak;
  if (inflight) *inflight = (int32_t)s->running.size();
  if (queued) *queued = (int32_t)s->queue.size();
  if (resident) *resident = (int32_t)s->resident.size();
  return ABF_OK;
}

abf_status abf_server_destroy(abf_server s) {
  if (!s) return ABF_ERR_INVALID;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
    s->paused = false;
  }
  s->cv_work.notify_one();
  if (s->worker.joinable()) s->worker.join();
  cudaSetDevice(s->device);
  for (auto& r : s->resident) cudaFree(r.d_g);
  for (auto& kv : s->plans) abf_plan_destroy(kv.second);
  for (auto& kv : s->jobs) delete kv.second;
  for (auto st : s->streams) {
    cudaStreamSynchronize(st);
    cudaStreamDestroy(st);
  }
  if (s->h_dev_status) cudaFreeHost(s->h_dev_status);
  if (s->d_slot_status) cudaFree(s->d_slot_status);
  if (s->d_slot_counter) cudaFree(s->d_slot_counter);
  if (s->base_ev) cudaEventDestroy(s->base_ev);
  delete s;
  return ABF_OK;
}

}  // extern "C"
