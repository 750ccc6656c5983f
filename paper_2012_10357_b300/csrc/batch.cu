// Batched requests: the C ABI of the wavefront path (pr_batch_*, pr_trace_batch*).
//
// A batch object owns the device memory of one batched launch (request table,
// per-pixel state, ray queues) sized for max_requests / max_pixels, a pinned
// staging copy of the request table, and a CUDA graph of the stage sequence.
// The kernels read the batch's request count and totals from device memory,
// so one captured graph serves every batch that fits the capacity.
#include <cuda_runtime.h>

#include <algorithm>
#include <string>
#include <vector>

#include "../../include/proceduray.h"
#include "internal.h"
#include "wavefront.h"

using namespace pr;

struct pr_batch {
  uint32_t max_req = 0;
  uint64_t max_px = 0;
  char* arena = nullptr;
  size_t arena_bytes = 0;
  BatchView V{};
  char* staging = nullptr;            // pinned: BatchHdr followed by ReqDev[max_req]
  cudaEvent_t staged = nullptr;       // the last staging copy has been consumed
  BatchTuning tuning{8, 16, 8, 64, 0};
  int n_sm = 0;
  cudaStream_t capture_stream = nullptr;
  // Captured launches, one per kernel family: batches with and without a
  // mirror-ray request (a server's iterations alternate between the two).
  struct Graph {
    cudaGraphExec_t exec = nullptr;
    BatchTuning tuning{};
    uint32_t tiles = 0;              // grid of the captured one-CTA-per-tile megakernel
    uint32_t launches = 0;
    bool ahs = false;
  } graphs[2];
  uint32_t staged_tiles = 0;         // tiles of the last staged batch
  BatchTuning staged_tuning{};       // launch shape the last staged batch was laid out for
  bool staged_ahs = false;           // the last staged batch needs the any-hit march
  bool staged_mirror = true;         // the last staged batch has a request with mirror rays
  uint32_t last_launches = 0;
  uint32_t* notify = nullptr;        // completion flags for the next staged batch (host-mapped)
  uint32_t notify_seq = 0;
};

namespace {

pr_status bfail(pr_status st, const std::string& m) {
  pr_internal_set_error(m);
  return st;
}

pr_status bcuda(cudaError_t e, const char* what) {
  pr_internal_set_error(std::string(what) + ": " + cudaGetErrorString(e));
  return e == cudaErrorMemoryAllocation ? PR_ERR_OUT_OF_MEMORY : PR_ERR_CUDA;
}

size_t a256(size_t x) { return (x + 255) & ~(size_t)255; }

bool tuning_ok(const BatchTuning& t) {
  bool tile = (t.tile_w == 16 && t.tile_h == 8) || (t.tile_w == 32 && t.tile_h == 4) || (t.tile_w == 8 && t.tile_h == 16);
  if (t.megakernel > 4 ||
      ((t.megakernel == 1 || t.megakernel == 2 || t.megakernel == 4) && !(t.tile_w == 16 && t.tile_h == 8)))
    return false;
  return tile && t.ctas_per_sm >= 1 && t.ctas_per_sm <= 16 && t.queue_chunk >= 32 && t.queue_chunk <= 1024 &&
         t.queue_chunk % 32 == 0;
}

// Validate the requests and write the request table into the pinned staging
// buffer, then copy it to the device on `st`.
pr_status stage(pr_batch* b, uint32_t n, const pr_request* reqs, uint64_t* counter, cudaStream_t st) {
  if (n == 0 || n > b->max_req) return bfail(PR_ERR_INVALID_ARG, "request count outside 1..max_requests");
  if (!reqs) return bfail(PR_ERR_INVALID_ARG, "null request array");
  // the previous staging copy must have been consumed before it is overwritten
  cudaError_t e = cudaEventSynchronize(b->staged);
  if (e != cudaSuccess) return bcuda(e, "wait for staging buffer");
  BatchHdr* H = reinterpret_cast<BatchHdr*>(b->staging);
  ReqDev* R = reinterpret_cast<ReqDev*>(b->staging + a256(sizeof(BatchHdr)));
  // A scene with an any-hit shader on a sphere-traced shader takes the batch
  // to the megakernel compiled with the any-hit march (16x8 tiles).
  bool ahs = false;
  for (uint32_t i = 0; i < n; ++i) ahs = ahs || pr_internal_ahs_march(reqs[i].scene);
  BatchTuning T = b->tuning;
  if (ahs) {
    T.tile_w = 16;
    T.tile_h = 8;
    T.megakernel = 2;
  }
  uint64_t px = 0;
  uint32_t tiles = 0;
  bool mirror = false;
  for (uint32_t i = 0; i < n; ++i) {
    const pr_request& q = reqs[i];
    mirror = mirror || q.params.max_depth >= 2;
    const pr_trace_params& p = q.params;
    if (!q.scene || !pr_internal_built(q.scene)) return bfail(PR_ERR_NOT_BUILT, "request scene null or not built");
    if (!q.out_rgba) return bfail(PR_ERR_INVALID_ARG, "request output null");
    if (p.struct_size != sizeof(pr_trace_params) || p.width == 0 || p.height == 0 || p.width > 65536 ||
        p.height > 65536 || p.max_depth < 1 || p.max_depth > 2 || p.max_steps == 0 || (p.flags & PR_TRACE_WRITE_AOV))
      return bfail(PR_ERR_INVALID_ARG, "bad request params (AOV output is not available in batches)");
    ReqDev& d = R[i];
    d.S = pr_internal_view(q.scene);
    d.cam = camera_frame(q.camera, p.width, p.height);
    d.light = make_float3(p.light_pos[0], p.light_pos[1], p.light_pos[2]);
    d.background = make_float3(p.background[0], p.background[1], p.background[2]);
    d.light_intensity = p.light_intensity;
    d.eps_rel = p.eps_rel;
    d.ambient = p.ambient;
    d.width = p.width;
    d.height = p.height;
    d.max_depth = p.max_depth;
    d.max_steps = p.max_steps;
    const uint32_t rows = q.row_count ? q.row_count : p.height;
    if ((q.row_count == 0 && q.row_begin != 0) || (uint64_t)q.row_begin + rows > p.height)
      return bfail(PR_ERR_INVALID_ARG, "request rows outside the image");
    d.row_begin = q.row_begin;
    d.rows = rows;
    d.tile_begin = tiles;
    d.tiles_x = (p.width + T.tile_w - 1) / T.tile_w;
    d.out = reinterpret_cast<float4*>(q.out_rgba);
    d.out_rgb = (p.flags & PR_TRACE_OUTPUT_RGB) ? 1u : 0u;
    d.tiles_done = 0u;
    d.pad_[0] = d.pad_[1] = d.pad_[2] = 0u;
    d.pixel_begin = px;
    uint64_t t = (uint64_t)d.tiles_x * ((rows + T.tile_h - 1) / T.tile_h);
    if (tiles + t > 0xFFFFFFFFull) return bfail(PR_ERR_INVALID_ARG, "too many tiles");
    d.n_tiles = (uint32_t)t;
    tiles += (uint32_t)t;
    px += (uint64_t)p.width * rows;
  }
  if (px > b->max_px) return bfail(PR_ERR_BUDGET, "batch pixels exceed the batch's max_pixels");
  H->n_req = n;
  H->total_tiles = tiles;
  b->staged_tiles = tiles;
  b->staged_tuning = T;
  b->staged_ahs = ahs;
  b->staged_mirror = mirror;
  H->total_pixels = px;
  H->tile_ctr = H->shadow_n = H->mirror_n = H->shadow_ctr = H->mirror_ctr = H->pad = 0;
  H->counter = reinterpret_cast<unsigned long long*>(counter);
  H->notify = b->notify;
  H->seq = b->notify_seq;
  H->pad2 = 0;
  H->job_n[0] = H->job_n[1] = H->job_ctr[0] = H->job_ctr[1] = 0;
  H->shade_ctr = H->finish_ctr = H->pad3[0] = H->pad3[1] = 0;
  b->notify = nullptr;   // one batch only
  size_t bytes = a256(sizeof(BatchHdr)) + sizeof(ReqDev) * n;
  e = cudaMemcpyAsync(b->V.hdr, b->staging, bytes, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaEventRecord(b->staged, st);
  if (e != cudaSuccess) return bcuda(e, "copy request table");
  return PR_OK;
}

pr_status capture(pr_batch* b, pr_batch::Graph& G) {
  if (G.exec) {
    cudaGraphExecDestroy(G.exec);
    G.exec = nullptr;
  }
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamBeginCapture(b->capture_stream, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return bcuda(e, "begin capture");
  G.launches = (uint32_t)launch_wavefront(b->V, b->staged_tuning, b->n_sm, G.tiles, b->capture_stream, b->staged_ahs,
                                          b->staged_mirror);
  e = cudaStreamEndCapture(b->capture_stream, &g);
  if (e != cudaSuccess) return bcuda(e, "end capture");
  e = cudaGraphInstantiate(&G.exec, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    G.exec = nullptr;
    return bcuda(e, "instantiate graph");
  }
  G.tuning = b->staged_tuning;
  G.ahs = b->staged_ahs;
  return PR_OK;
}

}  // namespace

extern "C" {

pr_status pr_batch_create(uint32_t max_requests, uint64_t max_pixels, pr_batch** out) {
  if (!out || max_requests == 0 || max_requests > (1u << 20) || max_pixels == 0 || max_pixels > (1ull << 32))
    return bfail(PR_ERR_INVALID_ARG, "pr_batch_create: need out, 1 <= max_requests <= 2^20, 1 <= max_pixels <= 2^32");
  *out = nullptr;
  pr_batch* b = new pr_batch();
  b->max_req = max_requests;
  b->max_px = max_pixels;
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&b->n_sm, cudaDevAttrMultiProcessorCount, dev);
  const uint64_t P = max_pixels;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t o = off;
    off = a256(off + bytes);
    return o;
  };
  size_t o_hdr = take(a256(sizeof(BatchHdr)) + sizeof(ReqDev) * max_requests);
  size_t o_sta = take(16 * P), o_stb = take(8 * P), o_refl = take(16 * P);
  size_t o_sqa = take(16 * P), o_sqb = take(16 * P), o_sqp = take(8 * P), o_sqr = take(4 * P);
  size_t o_mqa = take(16 * P), o_mqb = take(16 * P), o_mqp = take(8 * P), o_mqr = take(4 * P);
  // regrouped mode: traversal results per ray slot, march jobs
  // (one job per pixel per pass; rays beyond that march in place)
  size_t o_rgh = take(16 * P), o_rgj = take(8 * P), o_rgmh = take(16 * P), o_rgmj = take(8 * P),
         o_rgsj = take(8 * P);
  const uint64_t job_cap = (P + 1) / 2;   // jobs per pass; rays beyond march in place
  size_t o_job[2][2];
  for (int pass = 0; pass < 2; ++pass) {
    o_job[pass][0] = take(16 * kJobRows * job_cap);
    o_job[pass][1] = take(16 * job_cap);
  }
  b->arena_bytes = off;
  cudaError_t e = cudaMalloc(&b->arena, off);
  if (e != cudaSuccess) {
    delete b;
    return bcuda(e, "cudaMalloc batch arena");
  }
  char* A = b->arena;
  b->V.hdr = reinterpret_cast<BatchHdr*>(A + o_hdr);
  b->V.reqs = reinterpret_cast<const ReqDev*>(A + o_hdr + a256(sizeof(BatchHdr)));
  b->V.st_a = reinterpret_cast<float4*>(A + o_sta);
  b->V.st_b = reinterpret_cast<uint2*>(A + o_stb);
  b->V.refl = reinterpret_cast<float4*>(A + o_refl);
  b->V.sq_a = reinterpret_cast<float4*>(A + o_sqa);
  b->V.sq_b = reinterpret_cast<float4*>(A + o_sqb);
  b->V.sq_px = reinterpret_cast<uint64_t*>(A + o_sqp);
  b->V.sq_req = reinterpret_cast<uint32_t*>(A + o_sqr);
  b->V.mq_a = reinterpret_cast<float4*>(A + o_mqa);
  b->V.mq_b = reinterpret_cast<float4*>(A + o_mqb);
  b->V.mq_px = reinterpret_cast<uint64_t*>(A + o_mqp);
  b->V.mq_req = reinterpret_cast<uint32_t*>(A + o_mqr);
  b->V.rg_hit = reinterpret_cast<int4*>(A + o_rgh);
  b->V.rg_jobs = reinterpret_cast<uint2*>(A + o_rgj);
  b->V.rg_mhit = reinterpret_cast<int4*>(A + o_rgmh);
  b->V.rg_mjobs = reinterpret_cast<uint2*>(A + o_rgmj);
  b->V.rg_sjobs = reinterpret_cast<uint2*>(A + o_rgsj);
  for (int pass = 0; pass < 2; ++pass) {
    b->V.jobs[pass].a = reinterpret_cast<float4*>(A + o_job[pass][0]);
    b->V.jobs[pass].r = reinterpret_cast<float4*>(A + o_job[pass][1]);
  }
  b->V.job_cap = (uint32_t)job_cap;
  b->V.max_req = max_requests;
  e = cudaMallocHost(&b->staging, a256(sizeof(BatchHdr)) + sizeof(ReqDev) * max_requests);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->staged, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->capture_stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventRecord(b->staged, b->capture_stream);
  if (e != cudaSuccess) {
    pr_batch_destroy(b);
    return bcuda(e, "batch host staging / stream");
  }
  *out = b;
  return PR_OK;
}

pr_status pr_batch_set_tuning(pr_batch* b, const pr_batch_tuning* t) {
  if (!b || !t || t->struct_size != sizeof(pr_batch_tuning)) return bfail(PR_ERR_INVALID_ARG, "null batch/tuning or size");
  BatchTuning bt{t->ctas_per_sm, t->tile_w, t->tile_h, t->queue_chunk, t->megakernel};
  if (!tuning_ok(bt))
    return bfail(PR_ERR_INVALID_ARG, "tuning: tiles 16x8, 32x4 or 8x16; 1..16 CTAs/SM; chunk multiple of 32 in 32..1024");
  if (bt.megakernel == 3 && b->max_px >= (1ull << 31))
    return bfail(PR_ERR_INVALID_ARG, "the regrouped mode takes batches of fewer than 2^31 pixels");
  b->tuning = bt;
  return PR_OK;
}

pr_status pr_batch_get_tuning(const pr_batch* b, pr_batch_tuning* t) {
  if (!b || !t) return bfail(PR_ERR_INVALID_ARG, "null batch/tuning");
  t->struct_size = sizeof(pr_batch_tuning);
  t->ctas_per_sm = b->tuning.ctas_per_sm;
  t->tile_w = b->tuning.tile_w;
  t->tile_h = b->tuning.tile_h;
  t->queue_chunk = b->tuning.queue_chunk;
  t->megakernel = b->tuning.megakernel;
  return PR_OK;
}

pr_status pr_trace_batch(pr_batch* b, uint32_t n, const pr_request* reqs, uint64_t* ray_counter, void* stream) {
  if (!b) return bfail(PR_ERR_INVALID_ARG, "null batch");
  cudaStream_t st = (cudaStream_t)stream;
  pr_status s = stage(b, n, reqs, ray_counter, st);
  if (s != PR_OK) return s;
  b->last_launches = (uint32_t)launch_wavefront(b->V, b->staged_tuning, b->n_sm, b->staged_tiles, st, b->staged_ahs,
                                                b->staged_mirror);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return bcuda(e, "wavefront launch");
  return PR_OK;
}

pr_status pr_trace_batch_graph(pr_batch* b, uint32_t n, const pr_request* reqs, uint64_t* ray_counter, void* stream) {
  if (!b) return bfail(PR_ERR_INVALID_ARG, "null batch");
  cudaStream_t st = (cudaStream_t)stream;
  pr_status s = stage(b, n, reqs, ray_counter, st);
  if (s != PR_OK) return s;
  // the one-CTA-per-tile megakernel needs a grid of at least this batch's tiles: capture again
  // (with room to grow) when it is larger than the captured one
  pr_batch::Graph& G = b->graphs[b->staged_mirror ? 1 : 0];
  const bool grow = (b->staged_tuning.megakernel == 2 || b->staged_tuning.megakernel == 4) && b->staged_tiles > G.tiles;
  if (grow) {
    uint32_t g = 1024;
    while (g < b->staged_tiles && g < 0x80000000u) g <<= 1;
    G.tiles = g;
  }
  if (!G.exec || grow || G.ahs != b->staged_ahs || memcmp(&G.tuning, &b->staged_tuning, sizeof(BatchTuning)) != 0) {
    pr_status c = capture(b, G);
    if (c != PR_OK) return c;
  }
  cudaError_t e = cudaGraphLaunch(G.exec, st);
  if (e != cudaSuccess) return bcuda(e, "graph launch");
  b->last_launches = G.launches;
  return PR_OK;
}

pr_status pr_batch_autotune(pr_batch* b, uint32_t n, const pr_request* reqs, void* stream, pr_batch_tuning* best,
                            float* best_ms) {
  if (!b || !best) return bfail(PR_ERR_INVALID_ARG, "null batch/output");
  cudaStream_t st = (cudaStream_t)stream;
  const uint32_t ctas[] = {2, 4, 8, 12, 16};
  const uint32_t tiles[][2] = {{16, 8}, {32, 4}, {8, 16}};
  const uint32_t chunks[] = {32, 128};
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  BatchTuning keep = b->tuning, win = b->tuning;
  float win_ms = 1e30f;
  pr_status status = PR_OK;
  // the wavefront shapes, then the megakernel at 4 and 8 CTAs per SM (16x8 tiles)
  std::vector<BatchTuning> cands;
  for (uint32_t c : ctas)
    for (auto& tw : tiles)
      for (uint32_t ch : chunks) cands.push_back(BatchTuning{c, tw[0], tw[1], ch, 0u});
  cands.push_back(BatchTuning{4, 16, 8, 32, 1u});
  cands.push_back(BatchTuning{8, 16, 8, 32, 1u});
  cands.push_back(BatchTuning{4, 16, 8, 32, 2u});
  cands.push_back(BatchTuning{4, 16, 8, 32, 4u});
  // the regrouped stages (fractal marches from a job queue)
  if (b->max_px < (1ull << 31))
    for (uint32_t c : {4u, 8u})
      for (uint32_t ch : {32u, 128u}) cands.push_back(BatchTuning{c, 16, 8, ch, 3u});
  for (const BatchTuning& cand : cands) {
    b->tuning = cand;
    float ms_best = 1e30f;
    for (int rep = 0; rep < 3 && status == PR_OK; ++rep) {
      cudaEventRecord(e0, st);
      status = pr_trace_batch(b, n, reqs, nullptr, st);
      cudaEventRecord(e1, st);
      cudaEventSynchronize(e1);
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (rep > 0) ms_best = std::min(ms_best, ms);   // first run warms caches
    }
    if (status != PR_OK) break;
    if (ms_best < win_ms) {
      win_ms = ms_best;
      win = b->tuning;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  b->tuning = status == PR_OK ? win : keep;
  if (status != PR_OK) return status;
  best->struct_size = sizeof(pr_batch_tuning);
  best->ctas_per_sm = win.ctas_per_sm;
  best->tile_w = win.tile_w;
  best->tile_h = win.tile_h;
  best->queue_chunk = win.queue_chunk;
  best->megakernel = win.megakernel;
  if (best_ms) *best_ms = win_ms;
  return PR_OK;
}

size_t pr_batch_device_bytes(const pr_batch* b) { return b ? b->arena_bytes : 0; }

}  // extern "C"

bool pr_internal_batch_notify(pr_batch* b, uint32_t* notify, uint32_t seq) {
  if (!b || b->tuning.megakernel == 0) return false;
  b->notify = notify;
  b->notify_seq = seq;
  return true;
}

extern "C" {

void pr_batch_destroy(pr_batch* b) {
  if (!b) return;
  cudaDeviceSynchronize();
  for (auto& G : b->graphs)
    if (G.exec) cudaGraphExecDestroy(G.exec);
  if (b->capture_stream) cudaStreamDestroy(b->capture_stream);
  if (b->staged) cudaEventDestroy(b->staged);
  if (b->staging) cudaFreeHost(b->staging);
  if (b->arena) cudaFree(b->arena);
  delete b;
}

}  // extern "C"
