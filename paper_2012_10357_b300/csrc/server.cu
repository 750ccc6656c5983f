// Serving loop (pr_server_*): render requests arrive at any time; a worker
// thread admits them by a device-memory budget, keeps their scenes (device
// BVH) resident in a cache keyed by the caller's scene key, and renders
// with continuous batching: every iteration is one batched wavefront launch
// over row ranges of all admitted requests, so requests that arrive while
// others are on the GPU join at the next iteration and their work overlaps
// (under light load, solo_max_waiting requests or fewer waiting, the oldest
// runs alone through pr_trace).
// PR_SERVE_PLAIN mode renders one whole request per pr_trace, first come
// first served, for comparison.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <list>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <unordered_set>
#include <vector>

#include "../../include/proceduray.h"
#include "internal.h"

namespace {

double now_s() {
  using namespace std::chrono;
  return duration<double>(steady_clock::now().time_since_epoch()).count();
}

// Deep copy of a scene description (the caller's arrays may be freed after submit).
struct DescCopy {
  pr_scene_desc d{};
  std::vector<float> aabbs, params, xform, materials;
  std::vector<uint32_t> gpb, gpc, bgb, bgc, iblas, iid, isbt, imask, hg, sbt, rt, gtype, idx;
  std::vector<float> verts;
  explicit DescCopy(const pr_scene_desc* s) {
    d = *s;
    auto cpf = [](std::vector<float>& v, const float* p, size_t n) { v.assign(p, p + (p ? n : 0)); return v.data(); };
    auto cpu = [](std::vector<uint32_t>& v, const uint32_t* p, size_t n) {
      v.assign(p, p + (p ? n : 0));
      return v.data();
    };
    d.aabbs = cpf(aabbs, s->aabbs, 6 * (size_t)s->n_prims);
    d.params = cpf(params, s->params, PR_PARAMS_PER_PRIM * (size_t)s->n_prims);
    d.inst_xform = cpf(xform, s->inst_xform, 12 * (size_t)s->n_inst);
    d.materials = cpf(materials, s->materials, 4 * (size_t)s->n_materials);
    d.geom_prim_begin = cpu(gpb, s->geom_prim_begin, s->n_geoms);
    d.geom_prim_count = cpu(gpc, s->geom_prim_count, s->n_geoms);
    d.blas_geom_begin = cpu(bgb, s->blas_geom_begin, s->n_blas);
    d.blas_geom_count = cpu(bgc, s->blas_geom_count, s->n_blas);
    d.inst_blas = cpu(iblas, s->inst_blas, s->n_inst);
    d.inst_id = cpu(iid, s->inst_id, s->n_inst);
    d.inst_sbt_offset = cpu(isbt, s->inst_sbt_offset, s->n_inst);
    d.inst_mask = cpu(imask, s->inst_mask, s->n_inst);
    d.hit_groups = cpu(hg, s->hit_groups, 3 * (size_t)s->n_hit_groups);
    d.sbt = cpu(sbt, s->sbt, 4 * (size_t)s->n_records);
    d.ray_types = cpu(rt, s->ray_types, 2 * (size_t)s->n_ray_types);
    d.geom_type = s->geom_type ? cpu(gtype, s->geom_type, s->n_geoms) : nullptr;
    d.vertices = cpf(verts, s->vertices, 3 * (size_t)s->n_vertices);
    d.indices = cpu(idx, s->indices, 3 * (size_t)s->n_triangles);
  }
};

struct CachedScene {
  pr_scene* scene = nullptr;   // null while the loader builds it
  size_t bytes = 0;            // device bytes (the plan's estimate while loading)
  int refs = 0;                // admitted requests using it
  double last_use = 0.0;
  bool ready = false;
};

struct Job {
  uint64_t ticket = 0;
  uint64_t key = 0;
  std::shared_ptr<DescCopy> desc;   // only when the key was not cached at submit time
  size_t bytes = 0;                 // device bytes its scene needs (from the description)
  size_t input_bytes = 0;           // bytes of its scene's inputs (the staging copy)
  pr_camera camera{};
  pr_trace_params params{};
  float* out = nullptr;
  uint32_t next_row = 0;
  uint32_t rows_inflight = 0, rows_finished = 0;
  pr_request_stats st{};
  bool loaded_for_me = false;       // the loader built the scene for this request
};

// One launch: the row ranges it renders, by position in the launch's request table.
struct Part {
  uint64_t ticket;
  uint32_t rows;
  bool done;
};

struct Iteration {
  cudaEvent_t done = nullptr;
  uint32_t seq = 0;
  bool flags = false;        // the kernel writes per-request completion flags
  std::vector<Part> parts;
};

}  // namespace

struct pr_server {
  pr_server_config cfg{};
  int device = 0;
  cudaStream_t stream = nullptr;        // launches
  cudaStream_t load_stream = nullptr;   // scene uploads and BVH builds
  pr_batch* batch = nullptr;
  size_t batch_bytes = 0;
  unsigned long long* d_rays = nullptr;
  uint32_t* notify = nullptr;           // host-mapped completion flags [max_active]
  char* staging = nullptr;              // pinned buffer the loader sends scene inputs through
  size_t staging_bytes = 0;
  uint32_t seq = 0;
  std::thread worker, loader;
  std::mutex mu;
  std::condition_variable cv, cv_done, cv_load;
  bool stop = false;
  std::deque<std::shared_ptr<Job>> pending;
  std::list<std::shared_ptr<Job>> active;
  std::unordered_map<uint64_t, std::shared_ptr<Job>> jobs;   // every ticket (kept for polling)
  std::unordered_map<uint64_t, CachedScene> cache;
  size_t cache_bytes = 0;               // resident scenes + reservations of scenes being built
  uint64_t next_ticket = 1;
  uint64_t completed = 0, cache_hits = 0, cache_misses = 0, evictions = 0, iterations = 0, scene_loads = 0;
  std::deque<Iteration> inflight;
  std::vector<cudaEvent_t> free_events;
  std::string error;
  pr_status failed = PR_OK;
};

namespace {

pr_status sfail(pr_status st, const std::string& m) {
  pr_internal_set_error(m);
  return st;
}

cudaEvent_t take_event(pr_server* s) {
  if (!s->free_events.empty()) {
    cudaEvent_t e = s->free_events.back();
    s->free_events.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreateWithFlags(&e, cudaEventDisableTiming);
  return e;
}

void complete_job(pr_server* s, Job& j, pr_status status, double t) {
  j.st.status = status;
  j.st.t_done = t;
  ++s->completed;
  s->cv_done.notify_all();
  s->cv_load.notify_all();   // memory may have been freed for a waiting load
}

// A resident scene may be evicted when no admitted request uses it and no
// pending request waits for it (a scene built for a request that the worker
// has not admitted yet must stay, or two requests could take turns evicting
// each other's scene forever).
bool evictable(const CachedScene& c, uint64_t key, const std::unordered_set<uint64_t>& wanted) {
  return c.ready && c.refs == 0 && !wanted.count(key);
}

// Make room for `need` bytes under the budget by removing evictable resident
// scenes, least recently used first. The removed scenes are handed back to be
// destroyed without the lock. Called with the lock held; false if the budget
// cannot hold `need` even then (nothing is removed in that case).
bool make_room(pr_server* s, size_t need, std::vector<pr_scene*>& victims) {
  std::unordered_set<uint64_t> wanted;
  for (auto& p : s->pending) wanted.insert(p->key);
  size_t freeable = 0;
  for (auto& kv : s->cache)
    if (evictable(kv.second, kv.first, wanted)) freeable += kv.second.bytes;
  if (s->cache_bytes - freeable + s->batch_bytes + need > s->cfg.mem_budget_bytes) return false;
  while (s->cache_bytes + s->batch_bytes + need > s->cfg.mem_budget_bytes) {
    auto victim = s->cache.end();
    for (auto it = s->cache.begin(); it != s->cache.end(); ++it)
      if (evictable(it->second, it->first, wanted) &&
          (victim == s->cache.end() || it->second.last_use < victim->second.last_use))
        victim = it;
    victims.push_back(victim->second.scene);
    s->cache_bytes -= victim->second.bytes;
    s->cache.erase(victim);
    ++s->evictions;
  }
  return true;
}

// Loader thread: builds the scenes of pending requests whose key is neither
// resident nor being built, oldest request first, on its own stream, so scene
// uploads and BVH builds never hold up the launches of admitted requests.
// The bytes a scene needs are known from its description, so the budget is
// checked (and room made) before anything is allocated.
void loader_main(pr_server* s) {
  cudaSetDevice(s->device);
  std::unique_lock<std::mutex> lk(s->mu);
  while (true) {
    if (s->stop && s->pending.empty()) break;
    std::shared_ptr<Job> j;
    for (auto& p : s->pending)
      if (p->desc && !s->cache.count(p->key)) {
        j = p;
        break;
      }
    if (!j) {
      s->cv_load.wait_for(lk, std::chrono::milliseconds(1));
      continue;
    }
    std::vector<pr_scene*> victims;
    if (!make_room(s, j->bytes, victims)) {
      // room frees up when admitted requests finish, or when pending requests
      // whose scenes are resident are admitted and finish
      bool busy = !s->active.empty();
      for (auto& kv : s->cache) busy = busy || kv.second.refs > 0 || !kv.second.ready;
      for (auto& p : s->pending) busy = busy || (p != j && s->cache.count(p->key));
      if (!busy) {   // cannot fit even with every other scene evicted and nothing in flight
        s->pending.erase(std::find(s->pending.begin(), s->pending.end(), j));
        complete_job(s, *j, PR_ERR_BUDGET, now_s());
        continue;
      }
      s->cv_load.wait_for(lk, std::chrono::milliseconds(1));   // wait for requests to finish
      continue;
    }
    CachedScene& slot = s->cache[j->key];
    slot.bytes = j->bytes;
    slot.ready = false;
    s->cache_bytes += j->bytes;
    std::shared_ptr<DescCopy> desc = j->desc;
    const size_t input_bytes = j->input_bytes;
    j->st.t_load_start = now_s();
    lk.unlock();
    for (pr_scene* v : victims) pr_scene_destroy(v);
    pr_scene* sc = nullptr;
    pr_status st = PR_OK;
    if (input_bytes > s->staging_bytes) {   // one pinned staging buffer serves every load (grown when needed)
      const size_t want = std::max(input_bytes, s->staging_bytes * 3 / 2);
      if (s->staging) cudaFreeHost(s->staging);
      s->staging = nullptr;
      s->staging_bytes = 0;
      if (cudaMallocHost(&s->staging, want) == cudaSuccess) s->staging_bytes = want;
      else st = PR_ERR_OUT_OF_MEMORY;
    }
    if (st == PR_OK)
      st = pr_internal_scene_create_staged(&desc->d, s->load_stream, s->staging, s->staging_bytes, &sc);
    if (st == PR_OK) st = pr_build_bvh(sc, s->load_stream);
    if (st == PR_OK && cudaStreamSynchronize(s->load_stream) != cudaSuccess) st = PR_ERR_CUDA;
    const std::string msg = st == PR_OK ? std::string() : std::string(pr_last_error());
    lk.lock();
    ++s->scene_loads;
    j->st.t_load_end = now_s();
    auto it = s->cache.find(j->key);
    if (st != PR_OK) {
      s->cache_bytes -= it->second.bytes;
      s->cache.erase(it);
      auto pj = std::find(s->pending.begin(), s->pending.end(), j);
      if (pj != s->pending.end()) s->pending.erase(pj);
      complete_job(s, *j, st, now_s());
      lk.unlock();
      if (sc) pr_scene_destroy(sc);
      lk.lock();
      continue;
    }
    const size_t bytes = pr_scene_device_bytes(sc);
    s->cache_bytes = s->cache_bytes - it->second.bytes + bytes;
    it->second.scene = sc;
    it->second.bytes = bytes;
    it->second.ready = true;
    it->second.last_use = now_s();
    j->loaded_for_me = true;
    s->cv.notify_all();
  }
}

// Admit pending requests whose scene is resident, oldest first, while slots
// allow (a request whose scene is being built does not hold up later ones).
void admit(pr_server* s) {
  for (auto p = s->pending.begin(); p != s->pending.end() && s->active.size() < s->cfg.max_active;) {
    std::shared_ptr<Job> j = *p;
    auto it = s->cache.find(j->key);
    if (it == s->cache.end() && !j->desc) {   // cached at submit time but evicted since: cannot rebuild
      p = s->pending.erase(p);
      complete_job(s, *j, PR_ERR_BUDGET, now_s());
      continue;
    }
    if (it == s->cache.end() || !it->second.ready) {
      ++p;
      continue;
    }
    if (j->loaded_for_me) ++s->cache_misses;
    else ++s->cache_hits;
    it->second.refs++;
    it->second.last_use = now_s();
    j->desc.reset();
    j->st.t_admit = now_s();
    p = s->pending.erase(p);
    s->active.push_back(j);
  }
}

// A part of an iteration is rendered: account its rows; the request is done
// with its last rows.
void finish_part(pr_server* s, Part& part, double t) {
  part.done = true;
  auto jt = s->jobs.find(part.ticket);
  if (jt == s->jobs.end()) return;
  Job& j = *jt->second;
  j.rows_inflight -= part.rows;
  j.rows_finished += part.rows;
  if (j.rows_finished >= j.params.height) {
    auto c = s->cache.find(j.key);
    if (c != s->cache.end()) {
      c->second.refs--;
      c->second.last_use = t;
    }
    s->active.remove(jt->second);
    complete_job(s, j, PR_OK, t);
  }
}

// Completed work of the launches in flight: per-request completion flags of
// the batched megakernel (a request is done as soon as its last tile is, not
// at the end of the launch), then whole launches by their events. Stream
// order means that every launch before one that wrote a flag is complete, so
// a flag value at or past a launch's sequence number marks its part done.
void retire(pr_server* s) {
  const double t = now_s();
  for (Iteration& it : s->inflight) {
    if (!it.flags) continue;
    for (size_t k = 0; k < it.parts.size(); ++k) {
      Part& part = it.parts[k];
      if (part.done) continue;
      const uint32_t v = reinterpret_cast<volatile uint32_t*>(s->notify)[k];
      if ((int32_t)(v - it.seq) >= 0) finish_part(s, part, t);
    }
  }
  while (!s->inflight.empty() && cudaEventQuery(s->inflight.front().done) == cudaSuccess) {
    Iteration& it = s->inflight.front();
    for (Part& part : it.parts)
      if (!part.done) finish_part(s, part, t);
    s->free_events.push_back(it.done);
    s->inflight.pop_front();
  }
}

// One iteration: row ranges of active requests, oldest first, up to the pixel budget.
bool launch_iteration(pr_server* s) {
  std::vector<pr_request> reqs;
  Iteration it;
  uint64_t px = 0;
  const uint64_t cap = s->cfg.max_batch_pixels;
  const double t_launch = now_s();   // one time stamp for every request of this launch
  // Continuous batching pays when requests queue: with at most
  // solo_max_waiting requests waiting for rows, the oldest (whole, within the
  // pixel cap) runs alone through the single-request kernel, as in the plain
  // form (same image bits).
  bool single = s->cfg.mode == PR_SERVE_PLAIN;
  if (!single && s->cfg.solo_max_waiting) {
    uint32_t waiting = 0;
    const Job* first = nullptr;
    for (auto& jp : s->active) {
      if (jp->next_row >= jp->params.height) continue;
      if (!first) first = jp.get();
      ++waiting;
    }
    single = first && waiting <= s->cfg.solo_max_waiting && first->next_row == 0 &&
             (uint64_t)first->params.width * first->params.height <= cap;
  }
  for (auto& jp : s->active) {
    Job& j = *jp;
    if (j.next_row >= j.params.height) continue;
    if (reqs.size() >= s->cfg.max_active) break;
    uint64_t room = cap > px ? cap - px : 0;
    if (room < j.params.width) break;
    uint32_t rows = (uint32_t)std::min<uint64_t>(j.params.height - j.next_row, room / j.params.width);
    if (single) rows = j.params.height - j.next_row;
    pr_request r{};
    r.scene = s->cache[j.key].scene;
    r.camera = j.camera;
    r.params = j.params;
    r.out_rgba = j.out;
    r.row_begin = j.next_row;
    r.row_count = rows;
    reqs.push_back(r);
    if (j.st.t_first_launch == 0.0) j.st.t_first_launch = t_launch;
    j.next_row += rows;
    j.rows_inflight += rows;
    it.parts.push_back(Part{j.ticket, rows, false});
    px += (uint64_t)rows * j.params.width;
    if (single) break;   // one request per launch
  }
  if (reqs.empty()) return false;
  pr_status st;
  const bool whole_single = reqs.size() == 1 && reqs[0].row_begin == 0 && reqs[0].row_count == reqs[0].params.height;
  if (single || whole_single) {
    // plain form, or an iteration that is one whole request: the megakernel
    // (same image bits, one launch instead of the four batched stages)
    st = pr_trace(reqs[0].scene, &reqs[0].camera, &reqs[0].params, reqs[0].out_rgba, nullptr,
                  reinterpret_cast<uint64_t*>(s->d_rays), s->stream);
  } else {
    it.seq = ++s->seq;
    it.flags = pr_internal_batch_notify(s->batch, s->notify, it.seq);
    st = pr_trace_batch_graph(s->batch, (uint32_t)reqs.size(), reqs.data(), reinterpret_cast<uint64_t*>(s->d_rays),
                              s->stream);
  }
  if (st != PR_OK) {
    s->failed = st;
    s->error = pr_last_error();
    return false;
  }
  it.done = take_event(s);
  cudaEventRecord(it.done, s->stream);
  s->inflight.push_back(std::move(it));
  ++s->iterations;
  return true;
}

void worker_main(pr_server* s) {
  cudaSetDevice(s->device);
  std::unique_lock<std::mutex> lk(s->mu);
  while (true) {
    if (s->stop && s->pending.empty() && s->active.empty() && s->inflight.empty()) break;
    retire(s);
    admit(s);
    // keep up to two iterations queued on the stream so the GPU never idles
    bool launched = false;
    while (s->inflight.size() < 2 && s->failed == PR_OK) {
      if (!launch_iteration(s)) break;
      launched = true;
    }
    if (!launched) {
      if (!s->inflight.empty()) {
        lk.unlock();
        std::this_thread::sleep_for(std::chrono::microseconds(20));
        lk.lock();
      } else {
        s->cv.wait_for(lk, std::chrono::milliseconds(1));
      }
    }
  }
}

}  // namespace

extern "C" {

pr_status pr_server_create(const pr_server_config* cfg, pr_server** out) {
  if (!cfg || !out || cfg->struct_size != sizeof(pr_server_config))
    return sfail(PR_ERR_INVALID_ARG, "pr_server_create: null config/output or struct_size mismatch");
  if (cfg->max_active == 0 || cfg->max_batch_pixels == 0 ||
      (cfg->mode != PR_SERVE_CONTINUOUS && cfg->mode != PR_SERVE_PLAIN))
    return sfail(PR_ERR_INVALID_ARG, "pr_server_create: max_active, max_batch_pixels must be > 0; mode 0 or 1");
  *out = nullptr;
  pr_server* s = new pr_server();
  s->cfg = *cfg;
  cudaGetDevice(&s->device);
  cudaError_t e = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking);
  // scene uploads and BVH builds on the highest-priority stream: their kernels
  // are scheduled ahead of the rendering launches' waiting CTAs (measured on
  // B300 with a 1080p render running: a 100 000-instance scene load of 10-19 ms
  // at normal priority, about 5 ms at high priority)
  int prio_least = 0, prio_greatest = 0;
  if (e == cudaSuccess) e = cudaDeviceGetStreamPriorityRange(&prio_least, &prio_greatest);
  if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&s->load_stream, cudaStreamNonBlocking, prio_greatest);
  if (e == cudaSuccess) e = cudaHostAlloc(&s->notify, sizeof(uint32_t) * cfg->max_active, cudaHostAllocMapped);
  if (e == cudaSuccess) std::memset(s->notify, 0, sizeof(uint32_t) * cfg->max_active);
  if (e == cudaSuccess) e = cudaMalloc(&s->d_rays, sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaMemsetAsync(s->d_rays, 0, sizeof(unsigned long long), s->stream);
  if (e != cudaSuccess) {
    pr_server_destroy(s);
    return sfail(e == cudaErrorMemoryAllocation ? PR_ERR_OUT_OF_MEMORY : PR_ERR_CUDA,
                 std::string("pr_server_create: ") + cudaGetErrorString(e));
  }
  if (cfg->mode == PR_SERVE_CONTINUOUS) {
    pr_status st = pr_batch_create(cfg->max_active, cfg->max_batch_pixels, &s->batch);
    if (st != PR_OK) {
      pr_server_destroy(s);
      return st;
    }
    s->batch_bytes = pr_batch_device_bytes(s->batch);
    if (cfg->tuning.struct_size == sizeof(pr_batch_tuning)) {
      st = pr_batch_set_tuning(s->batch, &cfg->tuning);
      if (st != PR_OK) {
        pr_server_destroy(s);
        return st;
      }
    }
  }
  if (s->batch_bytes > cfg->mem_budget_bytes) {
    pr_server_destroy(s);
    return sfail(PR_ERR_BUDGET, "pr_server_create: the batch state alone exceeds the memory budget");
  }
  s->worker = std::thread(worker_main, s);
  s->loader = std::thread(loader_main, s);
  *out = s;
  return PR_OK;
}

pr_status pr_server_submit(pr_server* s, const pr_server_request* r, uint64_t* ticket) {
  if (!s || !r || !ticket || !r->out_rgba) return sfail(PR_ERR_INVALID_ARG, "pr_server_submit: null argument");
  const pr_trace_params& p = r->params;
  if (p.struct_size != sizeof(pr_trace_params) || p.width == 0 || p.height == 0 || p.width > 65536 ||
      p.height > 65536 || p.max_depth < 1 || p.max_depth > 2 || p.max_steps == 0 || (p.flags & PR_TRACE_WRITE_AOV) ||
      (uint64_t)p.width > s->cfg.max_batch_pixels)
    return sfail(PR_ERR_INVALID_ARG, "pr_server_submit: bad params (no AOV; width must fit max_batch_pixels)");
  auto j = std::make_shared<Job>();
  j->key = r->scene_key;
  j->camera = r->camera;
  j->params = p;
  j->out = r->out_rgba;
  std::unique_lock<std::mutex> lk(s->mu);
  if (s->failed != PR_OK) return sfail(s->failed, "server stopped after an error: " + s->error);
  if (!s->cache.count(r->scene_key)) {
    if (!r->desc) return sfail(PR_ERR_INVALID_ARG, "pr_server_submit: scene key not cached and no description");
    lk.unlock();
    size_t bytes = 0, input_bytes = 0;
    pr_status v = pr_internal_scene_bytes(r->desc, &bytes, &input_bytes);   // validates the description
    if (v != PR_OK) return v;
    auto dc = std::make_shared<DescCopy>(r->desc);
    lk.lock();
    j->desc = dc;
    j->bytes = bytes;
    j->input_bytes = input_bytes;
  }
  j->ticket = s->next_ticket++;
  j->st.t_submit = now_s();
  s->jobs[j->ticket] = j;
  s->pending.push_back(j);
  *ticket = j->ticket;
  s->cv.notify_all();
  s->cv_load.notify_all();
  return PR_OK;
}

pr_status pr_server_poll(pr_server* s, uint64_t ticket, int* done, pr_request_stats* stats) {
  if (!s || !done) return sfail(PR_ERR_INVALID_ARG, "pr_server_poll: null argument");
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->jobs.find(ticket);
  if (it == s->jobs.end()) return sfail(PR_ERR_INVALID_ARG, "pr_server_poll: unknown ticket");
  const Job& j = *it->second;
  *done = j.st.t_done > 0.0 ? 1 : 0;
  if (stats) {
    *stats = j.st;
    stats->cache_hit = (j.st.t_admit > 0.0 && !j.loaded_for_me) ? 1u : 0u;
  }
  return PR_OK;
}

pr_status pr_server_drain(pr_server* s, double timeout_s) {
  if (!s) return sfail(PR_ERR_INVALID_ARG, "pr_server_drain: null server");
  std::unique_lock<std::mutex> lk(s->mu);
  auto until = std::chrono::steady_clock::now() + std::chrono::duration<double>(timeout_s);
  while (s->completed < s->next_ticket - 1 && s->failed == PR_OK) {
    if (s->cv_done.wait_until(lk, until) == std::cv_status::timeout &&
        s->completed < s->next_ticket - 1)
      return sfail(PR_ERR_TIMEOUT, "pr_server_drain: requests still in flight at the timeout");
  }
  if (s->failed != PR_OK) return sfail(s->failed, "server stopped after an error: " + s->error);
  return PR_OK;
}

pr_status pr_server_get_stats(pr_server* s, pr_server_stats* out) {
  if (!s || !out) return sfail(PR_ERR_INVALID_ARG, "pr_server_get_stats: null argument");
  unsigned long long rays = 0;
  cudaError_t e = cudaMemcpyAsync(&rays, s->d_rays, sizeof(rays), cudaMemcpyDeviceToHost, s->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  if (e != cudaSuccess) return sfail(PR_ERR_CUDA, std::string("pr_server_get_stats: ") + cudaGetErrorString(e));
  std::lock_guard<std::mutex> lk(s->mu);
  out->struct_size = sizeof(pr_server_stats);
  out->submitted = s->next_ticket - 1;
  out->completed = s->completed;
  out->rays = rays;
  out->iterations = s->iterations;
  out->cache_hits = s->cache_hits;
  out->cache_misses = s->cache_misses;
  out->evictions = s->evictions;
  out->cache_bytes = s->cache_bytes;
  out->batch_bytes = s->batch_bytes;
  out->scene_loads = s->scene_loads;
  return PR_OK;
}

void pr_server_destroy(pr_server* s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
    if (s->failed != PR_OK) {   // abandon queued work after a failure
      s->pending.clear();
      s->active.clear();
    }
  }
  s->cv.notify_all();
  s->cv_load.notify_all();
  if (s->worker.joinable()) s->worker.join();
  if (s->loader.joinable()) s->loader.join();
  if (s->stream) cudaStreamSynchronize(s->stream);
  if (s->load_stream) cudaStreamSynchronize(s->load_stream);
  for (auto& it : s->inflight) cudaEventDestroy(it.done);
  for (cudaEvent_t e : s->free_events) cudaEventDestroy(e);
  for (auto& c : s->cache) pr_scene_destroy(c.second.scene);
  if (s->batch) pr_batch_destroy(s->batch);
  if (s->d_rays) cudaFree(s->d_rays);
  if (s->notify) cudaFreeHost(s->notify);
  if (s->staging) cudaFreeHost(s->staging);
  if (s->stream) cudaStreamDestroy(s->stream);
  if (s->load_stream) cudaStreamDestroy(s->load_stream);
  delete s;
}

}  // extern "C"
