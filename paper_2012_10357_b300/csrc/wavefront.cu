// Batched wavefront path: many render requests (each its own scene, camera
// and resolution) fused into one set of persistent kernels per bounce:
//   primary  : tiles of all requests, claimed from one atomic counter; ray
//              generation, closest-hit traversal, surface and light set-up;
//              shadow and mirror rays are appended to queues with warp-ballot
//              compaction (one atomic per warp), so later stages run full warps
//   shadow   : any-hit traversal of the compacted shadow queue
//   mirror   : closest-hit traversal + unshadowed shading of the mirror queue
//   resolve  : per pixel, the same composition as the megakernel
// Per-pixel arithmetic is the megakernel's (shared device functions in
// tracer.cuh), so both paths produce the same image bits.
#include <cuda_runtime.h>

#include <cstdint>

#include "internal.h"
#include "tracer.cuh"
#include "wavefront.h"

namespace pr {
namespace {

constexpr uint32_t kFull = 0xFFFFFFFFu;

__device__ __forceinline__ uint32_t find_request(const ReqDev* reqs, uint32_t n, uint32_t tile) {
  // last request whose tile_begin <= tile (tile_begin is increasing)
  uint32_t lo = 0, hi = n;
  while (hi - lo > 1) {
    uint32_t mid = (lo + hi) >> 1;
    if (reqs[mid].tile_begin <= tile) lo = mid;
    else hi = mid;
  }
  return lo;
}

__device__ __forceinline__ uint32_t find_request_px(const ReqDev* reqs, uint32_t n, uint64_t px) {
  uint32_t lo = 0, hi = n;
  while (hi - lo > 1) {
    uint32_t mid = (lo + hi) >> 1;
    if (reqs[mid].pixel_begin <= px) lo = mid;
    else hi = mid;
  }
  return lo;
}

// Warp-aggregated append: returns the slot of this lane (valid only if want).
__device__ __forceinline__ uint32_t warp_append(uint32_t* count, bool want) {
  const uint32_t lane = threadIdx.x & 31;
  uint32_t m = __ballot_sync(kFull, want);
  if (!m) return 0;
  uint32_t leader = __ffs(m) - 1;
  uint32_t base = 0;
  if (lane == leader) base = atomicAdd(count, (uint32_t)__popc(m));
  base = __shfl_sync(kFull, base, leader);
  return base + __popc(m & ((1u << lane) - 1u));
}

template <int TW, int TH>
__global__ void __launch_bounds__(128, 4) k_wf_primary(BatchView B) {
  static_assert(TW * TH == 128, "128-pixel tiles");
  __shared__ ReqDev sreq;
  __shared__ uint32_t s_tile, s_req;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  constexpr int WX = TW / 8;   // warps across (8x4 pixel sub-tile per warp)
  const int ox = (warp % WX) * 8 + (lane & 7), oy = (warp / WX) * 4 + (lane >> 3);
  PR_DECLARE_STACK(128);
  uint32_t last_req = kFull;
  for (;;) {
    if (threadIdx.x == 0) {
      uint32_t t = atomicAdd(&B.hdr->tile_ctr, 1u);
      s_tile = t;
      s_req = t < B.hdr->total_tiles ? find_request(B.reqs, B.hdr->n_req, t) : 0;
    }
    __syncthreads();
    const uint32_t tile = s_tile, r = s_req;
    if (tile >= B.hdr->total_tiles) break;
    if (r != last_req) {
      const uint32_t* src = reinterpret_cast<const uint32_t*>(B.reqs + r);
      uint32_t* dst = reinterpret_cast<uint32_t*>(&sreq);
      for (int i = threadIdx.x; i < (int)(sizeof(ReqDev) / 4); i += blockDim.x) dst[i] = src[i];
      __syncthreads();
      last_req = r;
    }
    const ReqDev& R = sreq;
    const uint32_t lt = tile - R.tile_begin;
    const int x = (int)(lt % R.tiles_x) * TW + ox, y = (int)R.row_begin + (int)(lt / R.tiles_x) * TH + oy;
    const bool valid = x < (int)R.width && y < (int)(R.row_begin + R.rows);
    bool need_s = false, need_m = false;
    float3 os = f3(0.f, 0.f, 0.f), ds = os, orr = os, dr = os;
    float smax = 0.f;
    uint64_t px = 0;
    if (valid) {
      const SceneView& S = R.S;
      const float3 eye = R.cam.eye;
      const float3 d = camera_ray(R.cam, x, y);
      const float eps = scene_eps(S, R.eps_rel);
      px = R.pixel_begin + (uint64_t)(y - (int)R.row_begin) * R.width + (uint64_t)x;
      Hit h;
      trace_typed<false>(S, eye, d, 0, 0.f, INFINITY, eps, R.max_steps, h, stack, nullptr);
      uint32_t flags = 0;
      float4 a = make_float4(0.f, 0.f, 0.f, 0.f);
      float ndl = 0.f;
      if (h.inst >= 0) {
        flags |= 1u;
        Surface sf = surface_at(S, h, eye, d, eps, nullptr);
        if (sf.chs == PR_CHS_LAMBERT) {
          flags |= 0x100u;
          const float3 pt = madd(eye, h.t, d);
          const float delta = is_sphere_traced(sf.is_id) ? 2.f * eps : eps;
          ndl = light_ndl(sf, R.light, pt);
          a = make_float4(sf.albedo.x, sf.albedo.y, sf.albedo.z, sf.kr);
          if (ndl > 0.f) {
            os = madd(pt, delta, sf.n);
            float3 ls = R.light - os;
            smax = len3(ls);
            ds = ls * (1.f / smax);
            need_s = true;
            flags |= 2u;
          }
          if (R.max_depth >= 2 && sf.kr > 0.f) {
            orr = madd(pt, delta, sf.n);
            dr = normalize3(d - sf.n * (2.f * dot3(d, sf.n)));
            need_m = true;
            flags |= 8u;
          }
        }
      }
      B.st_a[px] = a;
      B.st_b[px] = make_uint2(__float_as_uint(ndl), flags);
    }
    uint32_t qs = warp_append(&B.hdr->shadow_n, need_s);
    if (need_s) {
      B.sq_a[qs] = make_float4(os.x, os.y, os.z, smax);
      B.sq_b[qs] = make_float4(ds.x, ds.y, ds.z, 0.f);
      B.sq_px[qs] = px;
      B.sq_req[qs] = r;
    }
    uint32_t qm = warp_append(&B.hdr->mirror_n, need_m);
    if (need_m) {
      B.mq_a[qm] = make_float4(orr.x, orr.y, orr.z, 0.f);
      B.mq_b[qm] = make_float4(dr.x, dr.y, dr.z, 0.f);
      B.mq_px[qm] = px;
      B.mq_req[qm] = r;
    }
    unsigned long long* counter = B.hdr->counter;
    if (counter) {
      uint32_t rays = (valid ? 1u : 0u) + (need_s ? 1u : 0u) + (need_m ? 1u : 0u);
      uint32_t tot = __reduce_add_sync(kFull, rays);
      if (lane == 0 && tot) atomicAdd(counter, (unsigned long long)tot);
    }
    __syncthreads();
  }
}

// Queue stages: each warp pops `chunk` rays at a time (lanes take every 32nd).
__global__ void __launch_bounds__(128, 4) k_wf_shadow(BatchView B, uint32_t chunk) {
  const int lane = threadIdx.x & 31;
  PR_DECLARE_STACK(128);
  const uint32_t n = B.hdr->shadow_n;
  for (;;) {
    uint32_t base = 0;
    if (lane == 0) base = atomicAdd(&B.hdr->shadow_ctr, chunk);
    base = __shfl_sync(kFull, base, 0);
    if (base >= n) break;
    for (uint32_t i = base + lane; i < base + chunk && i < n; i += 32) {
      const ReqDev& R = B.reqs[B.sq_req[i]];
      float4 a = B.sq_a[i], b = B.sq_b[i];
      const float eps = scene_eps(R.S, R.eps_rel);
      Hit sh;
      trace_typed<false>(R.S, f3(a.x, a.y, a.z), f3(b.x, b.y, b.z), 1, 0.f, a.w, eps, R.max_steps, sh, stack, nullptr);
      if (sh.inst < 0) {
        uint64_t px = B.sq_px[i];
        B.st_b[px].y |= 4u;
      }
    }
  }
}

__global__ void __launch_bounds__(128, 4) k_wf_mirror(BatchView B, uint32_t chunk) {
  const int lane = threadIdx.x & 31;
  PR_DECLARE_STACK(128);
  const uint32_t n = B.hdr->mirror_n;
  for (;;) {
    uint32_t base = 0;
    if (lane == 0) base = atomicAdd(&B.hdr->mirror_ctr, chunk);
    base = __shfl_sync(kFull, base, 0);
    if (base >= n) break;
    for (uint32_t i = base + lane; i < base + chunk && i < n; i += 32) {
      const ReqDev& R = B.reqs[B.mq_req[i]];
      float4 a = B.mq_a[i], b = B.mq_b[i];
      const float3 orr = f3(a.x, a.y, a.z), dr = f3(b.x, b.y, b.z);
      const float eps = scene_eps(R.S, R.eps_rel);
      Hit rh;
      trace_typed<false>(R.S, orr, dr, 0, 0.f, INFINITY, eps, R.max_steps, rh, stack, nullptr);
      float3 lr;
      uint64_t px = B.mq_px[i];
      if (rh.inst >= 0) {
        Surface s2 = surface_at(R.S, rh, orr, dr, eps, nullptr);
        lr = s2.chs == PR_CHS_LAMBERT
                 ? lambert_rgb(s2.albedo, R.ambient, R.light_intensity, light_ndl(s2, R.light, madd(orr, rh.t, dr)), 1.f)
                 : f3(0.f, 0.f, 0.f);
        B.st_b[px].y |= 16u;
      } else {
        lr = miss_rgb(R.S, 0, R.background);
      }
      B.refl[px] = make_float4(lr.x, lr.y, lr.z, 0.f);
    }
  }
}

__global__ void __launch_bounds__(256) k_wf_resolve(BatchView B) {
  const uint64_t total = B.hdr->total_pixels;
  const uint32_t nreq = B.hdr->n_req;
  for (uint64_t px = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; px < total;
       px += (uint64_t)gridDim.x * blockDim.x) {
    const ReqDev& R = B.reqs[find_request_px(B.reqs, nreq, px)];
    uint2 sb = B.st_b[px];
    uint32_t flags = sb.y;
    float3 color;
    if (!(flags & 1u)) {
      color = miss_rgb(R.S, 0, R.background);
    } else if (!(flags & 0x100u)) {
      color = f3(0.f, 0.f, 0.f);
    } else {
      float4 a = B.st_a[px];
      float ndl = __uint_as_float(sb.x);
      float vis = (flags & 2u) ? ((flags & 4u) ? 1.f : 0.f) : 1.f;
      color = lambert_rgb(f3(a.x, a.y, a.z), R.ambient, R.light_intensity, ndl, vis);
      if (flags & 8u) {
        float4 lr = B.refl[px];
        color = mirror_mix(color, f3(lr.x, lr.y, lr.z), a.w);
      }
    }
    const uint64_t local = px - R.pixel_begin;
    const uint64_t row = R.row_begin + local / R.width, col = local % R.width;
    const uint64_t o = row * R.width + col;
    if (R.out_rgb) {
      float* f = reinterpret_cast<float*>(R.out) + 3 * o;
      f[0] = color.x;
      f[1] = color.y;
      f[2] = color.z;
    } else {
      R.out[o] = make_float4(color.x, color.y, color.z, 1.f);
    }
  }
}

// ---- regrouped stages ------------------------------------------------------
// Sphere tracing a fractal (Julia, Mandelbulb) takes from a few to hundreds
// of estimates per ray, so in the stages above a warp whose rays reach a
// fractal runs at the pace of its slowest march with most lanes idle. Here
// the traversals hand their fractal candidates on as march jobs (appended to
// one queue per pass with a warp prefix sum and one atomic per warp), and a
// persistent march kernel refills every lane that finishes its march with the
// next job (a warp ballot over the idle lanes claims as many jobs as there are
// idle lanes), computing the normal stencil of a hit in the same loop. The
// closest hit is then the least (t, instance, geometry, primitive) over the
// traversal's own hit and the job hits, the rule of the in-place traversal:
// a job's march interval only extends the in-place one, and any hit it finds
// beyond the in-place interval lies past the closest hit, so the images are
// the same bits as the megakernel's.

constexpr uint32_t kEmptyJob = 0xFFFFFFFFu;   // job slot left unused (its ray overflowed the queue)
constexpr uint32_t kMirrorSlot = 0x80000000u; // pass-1 ray slot of a mirror ray (else a shadow ray)

// Every lane of the warp calls this (n = 0 for lanes without candidates).
// Returns the ray's first job, or kEmptyJob when the pass's queue is full
// (the caller then marches its candidates in place).
__device__ __forceinline__ uint32_t append_jobs(const BatchView& B, int pass, const Deferred& dfr, uint32_t slot,
                                                uint32_t req, bool normal, float eps, uint32_t max_steps) {
  const uint32_t lane = threadIdx.x & 31;
  const uint32_t n = (uint32_t)dfr.n;
  uint32_t x = n;   // inclusive prefix sum over the warp
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(kFull, x, o);
    if ((int)lane >= o) x += y;
  }
  const uint32_t total = __shfl_sync(kFull, x, 31);
  if (total == 0) return kEmptyJob;
  uint32_t base = 0;
  if (lane == 31) base = atomicAdd(&B.hdr->job_n[pass], total);
  base = __shfl_sync(kFull, base, 31);
  const uint32_t first = base + x - n;
  const MarchJobs& J = B.jobs[pass];
  const bool fits = (uint64_t)first + n <= B.job_cap;
  for (uint32_t i = 0; i < n; ++i) {
    const uint32_t j = first + i;
    if (j >= B.job_cap) break;
    float4* row = J.a + (size_t)kJobRows * j;
    if (fits) {
      const float4* prm = reinterpret_cast<const float4*>(B.reqs[req].S.params) + 4 * (size_t)dfr.prim[i];
      row[0] = make_float4(dfr.oo[i].x, dfr.oo[i].y, dfr.oo[i].z, dfr.t_lo[i]);
      row[1] = make_float4(dfr.dd[i].x, dfr.dd[i].y, dfr.dd[i].z, dfr.t_hi[i]);
      row[2] = make_float4(__int_as_float(dfr.inst[i]), __int_as_float(dfr.leaf[i]),
                           __uint_as_float(dfr.is_id[i] | (normal ? 0x10000u : 0u)), __uint_as_float(slot));
      row[3] = make_float4(eps, __uint_as_float(max_steps), __uint_as_float(req), 0.f);
      row[4] = __ldg(prm);
      row[5] = __ldg(prm + 1);
      row[6] = __ldg(prm + 2);
    } else {
      row[2].z = __uint_as_float(kEmptyJob);
    }
  }
  return fits ? first : kEmptyJob;
}

// The candidates of a ray whose jobs did not fit, marched where they are, with
// the acceptance rule of the traversal; true when a candidate hit (any-hit
// rays stop at the first).
__device__ __noinline__ bool march_in_place(const SceneView& S, const Deferred& dfr, float eps, uint32_t max_steps,
                                            bool any_hit, Hit& h) {
  bool found = false;
  for (int i = 0; i < dfr.n; ++i) {
    const int k = dfr.inst[i];
    IsResult res;
    if (run_intersection<false>(dfr.is_id[i], PR_NONE, S.params + 4 * (size_t)dfr.prim[i], dfr.oo[i], dfr.dd[i],
                                safe_rcp(dfr.dd[i]), 0.f, dfr.t_lo[i],
                                dfr.t_hi[i], eps, max_steps, res, nullptr)) {
      const uint2 gq = __ldg(S.leaf_gq + dfr.leaf[i]);
      bool accept = res.t < h.t;
      if (!accept && res.t == h.t && h.inst >= 0) accept = key_less(k, gq, h.inst, __ldg(S.leaf_gq + (h.leaf & 0x3FFFFFFF)));
      if (accept) {
        h.t = res.t;
        h.inst = k;
        h.leaf = dfr.leaf[i];
        h.attr = res.attr;
        found = true;
        if (any_hit) return true;
      }
    }
  }
  return found;
}

// The closest hit over the traversal's own hit and the ray's march jobs;
// returns the winning job (its gradient serves the normal), or -1.
__device__ __forceinline__ int resolve_jobs(const SceneView& S, const MarchJobs& J, uint32_t first, uint32_t n, Hit& h) {
  int best = -1;
  for (uint32_t i = 0; i < n; ++i) {
    const float4 r = J.r[first + i];
    if (r.x < 0.f) continue;   // the march found no surface
    const float4 a = J.a[(size_t)kJobRows * (first + i) + 2];
    const int k = __float_as_int(a.x), leaf = __float_as_int(a.y);
    bool accept = r.x < h.t;
    if (!accept && r.x == h.t && h.inst >= 0)
      accept = key_less(k, __ldg(S.leaf_gq + leaf), h.inst, __ldg(S.leaf_gq + (h.leaf & 0x3FFFFFFF)));
    if (accept) {
      h.t = r.x;
      h.inst = k;
      h.leaf = leaf;
      h.attr = 1u;
      best = (int)(first + i);
    }
  }
  return best;
}

// Primary rays: tiles of all requests; traversal with fractal candidates
// deferred; the closest other hit and the ray's jobs are kept per pixel.
template <int TW, int TH>
__global__ void __launch_bounds__(128, 4) k_rg_primary(BatchView B) {
  static_assert(TW * TH == 128, "128-pixel tiles");
  __shared__ uint32_t s_tile, s_req;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  constexpr int WX = TW / 8;
  const int ox = (warp % WX) * 8 + (lane & 7), oy = (warp / WX) * 4 + (lane >> 3);
  PR_DECLARE_STACK(128);
  for (;;) {
    if (threadIdx.x == 0) {
      const uint32_t t = atomicAdd(&B.hdr->tile_ctr, 1u);
      s_tile = t;
      s_req = t < B.hdr->total_tiles ? find_request(B.reqs, B.hdr->n_req, t) : 0;
    }
    __syncthreads();
    const uint32_t tile = s_tile, r = s_req;
    if (tile >= B.hdr->total_tiles) break;
    const ReqDev& R = B.reqs[r];
    const uint32_t lt = tile - R.tile_begin;
    const int x = (int)(lt % R.tiles_x) * TW + ox, y = (int)R.row_begin + (int)(lt / R.tiles_x) * TH + oy;
    const bool valid = x < (int)R.width && y < (int)(R.row_begin + R.rows);
    Deferred dfr;
    dfr.n = 0;
    Hit h;
    uint64_t px = 0;
    float3 eye = f3(0.f, 0.f, 0.f), d = eye;
    float eps = 0.f;
    if (valid) {
      const CameraBasis& cb = R.cam;
      eye = cb.eye;
      d = camera_ray(cb, x, y);
      eps = scene_eps(R.S, R.eps_rel);
      px = R.pixel_begin + (uint64_t)(y - (int)R.row_begin) * R.width + (uint64_t)x;
      trace_typed<false, false, kStackDepth, true>(R.S, eye, d, 0, 0.f, INFINITY, eps, R.max_steps, h, stack, nullptr,
                                                   &dfr);
    }
    uint32_t first = append_jobs(B, 0, dfr, (uint32_t)px, r, true, eps, R.max_steps);
    if (valid) {
      if (first == kEmptyJob && dfr.n > 0) {
        march_in_place(R.S, dfr, eps, R.max_steps, false, h);
        dfr.n = 0;
      }
      B.rg_hit[px] = make_int4(__float_as_int(h.t), h.inst, h.leaf, (int)h.attr);
      B.rg_jobs[px] = make_uint2(first, (uint32_t)dfr.n);
    }
    unsigned long long* counter = B.hdr->counter;
    if (counter) {
      const uint32_t tot = __reduce_add_sync(kFull, valid ? 1u : 0u);
      if (lane == 0 && tot) atomicAdd(counter, (unsigned long long)tot);
    }
    __syncthreads();
  }
}

// Persistent march kernel with lane refill. A lane's state is one job: the
// object-space ray of its instance, the estimator's parameters, and the march
// position; a hit on a radiance ray goes on with the six stencil estimates of
// its normal. Every step evaluates the estimator once, at the march point or
// at a stencil point, from one call site. Idle lanes are refilled from the
// warp's pool once a quarter of the warp is idle (or all of it), so the
// warp's job loads are issued together rather than at almost every step.
// (Measured alternative: one fractal iteration per trip instead of one
// estimate, so that lanes whose estimate escapes early move on; slower on
// B300, 1.8 ms against 1.0 ms for the 1080p teaser, and the estimator
// compiled in that loop no longer gives the in-place loop's bits.)
__global__ void __launch_bounds__(128, 8) k_rg_march(BatchView B, int pass) {
  const uint32_t lane = threadIdx.x & 31;
  const uint32_t n = min(B.hdr->job_n[pass], B.job_cap);
  const MarchJobs J = B.jobs[pass];
  int job = -1;
  bool exhausted = false;
  // the warp's pool of claimed jobs [pool_next, pool_end): refilled kPoolJobs at
  // a time with one atomic (warp-uniform values)
  constexpr uint32_t kPoolJobs = 64;
  constexpr int kRefillIdle = 8;
  uint32_t pool_next = 0, pool_end = 0;
  uint32_t is_id = 0, phase = 0, steps = 0, max_steps = 0;
  bool normal = false;
  float t = 0.f, t_hi = 0.f, inv_len = 0.f, eps = 0.f, hstep = 0.f, gx = 0.f, gy = 0.f, gz = 0.f;
  float3 o = f3(0.f, 0.f, 0.f), d = o, ph = o;
  float4 p0 = make_float4(0.f, 0.f, 0.f, 0.f), p1 = p0, p2 = p0;
  for (;;) {
    const bool idle = job < 0;
    const uint32_t want = __ballot_sync(kFull, idle);
    const bool refill = want == kFull || __popc(want) >= kRefillIdle;
    if (refill && pool_next >= pool_end && !exhausted) {
      uint32_t base = 0;
      if (lane == 0) base = atomicAdd(&B.hdr->job_ctr[pass], kPoolJobs);
      base = __shfl_sync(kFull, base, 0);
      if (base + kPoolJobs >= n) exhausted = true;
      pool_next = min(base, n);
      pool_end = min(base + kPoolJobs, n);
    }
    if (refill && pool_next < pool_end) {
      const uint32_t take = min((uint32_t)__popc(want), pool_end - pool_next);
      const uint32_t rank = (uint32_t)__popc(want & ((1u << lane) - 1u));
      const uint32_t j = pool_next + rank;
      pool_next += take;
      if (idle && rank < take) {
        const float4* row = J.a + (size_t)kJobRows * j;
        const float4 a0 = row[0], a1 = row[1], a2 = row[2], a3 = row[3];
        p0 = row[4];
        p1 = row[5];
        p2 = row[6];
        const uint32_t z = __float_as_uint(a2.z);
        if (z != kEmptyJob) {
          o = f3(a0.x, a0.y, a0.z);
          d = f3(a1.x, a1.y, a1.z);
          t = a0.w;
          t_hi = a1.w;
          eps = a3.x;
          max_steps = __float_as_uint(a3.y);
          inv_len = rsqrtf(dot3(d, d));
          is_id = z & 0xFFFFu;
          normal = (z >> 16) != 0u;
          steps = 0;
          phase = 0;
          job = (int)j;
        }
      }
    }
    if (!__any_sync(kFull, job >= 0)) {
      if (exhausted && pool_next >= pool_end) break;
      continue;
    }
    if (job < 0) continue;
    // the march ends at the step cap or past the interval (the in-place loop's order)
    if (phase == 0 && (steps >= max_steps || t > t_hi)) {
      J.r[job] = make_float4(-1.f, 0.f, 0.f, 0.f);
      job = -1;
      continue;
    }
    // the point of this step: on the ray, or stencil point k (+h, -h along x, y, z)
    const int k = (int)phase - 1;
    const float sh = (k & 1) ? -hstep : hstep;
    const int ax = k >> 1;
    const float3 q = phase == 0 ? madd(o, t, d)
                                : f3(ax == 0 ? ph.x + sh : ph.x, ax == 1 ? ph.y + sh : ph.y, ax == 2 ? ph.z + sh : ph.z);
    const float v = fractal_de(is_id, p0, p1, p2, q);
    if (phase == 0) {
      const float dist = __fmul_rn(v, inv_len);
      if (dist < eps) {
        if (normal) {
          phase = 1;
          hstep = eps * len3(d);
          ph = q;
        } else {
          J.r[job] = make_float4(t, 0.f, 0.f, 0.f);
          job = -1;
        }
      } else {
        t += dist;
        ++steps;
      }
    } else {
      if (ax == 0) gx = (k & 1) ? gx - v : v;
      else if (ax == 1) gy = (k & 1) ? gy - v : v;
      else gz = (k & 1) ? gz - v : v;
      if (++phase == 7) {
        J.r[job] = make_float4(t, gx, gy, gz);
        job = -1;
      }
    }
  }
}

// Primary hits resolved over their jobs; closest-hit set-up as in k_wf_primary;
// shadow and mirror rays appended to their queues.
template <int TW, int TH>
__global__ void __launch_bounds__(128, 4) k_rg_shade(BatchView B) {
  __shared__ uint32_t s_tile, s_req;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  constexpr int WX = TW / 8;
  const int ox = (warp % WX) * 8 + (lane & 7), oy = (warp / WX) * 4 + (lane >> 3);
  for (;;) {
    if (threadIdx.x == 0) {
      const uint32_t t = atomicAdd(&B.hdr->shade_ctr, 1u);
      s_tile = t;
      s_req = t < B.hdr->total_tiles ? find_request(B.reqs, B.hdr->n_req, t) : 0;
    }
    __syncthreads();
    const uint32_t tile = s_tile, r = s_req;
    if (tile >= B.hdr->total_tiles) break;
    const ReqDev& R = B.reqs[r];
    const uint32_t lt = tile - R.tile_begin;
    const int x = (int)(lt % R.tiles_x) * TW + ox, y = (int)R.row_begin + (int)(lt / R.tiles_x) * TH + oy;
    const bool valid = x < (int)R.width && y < (int)(R.row_begin + R.rows);
    bool need_s = false, need_m = false;
    float3 os = f3(0.f, 0.f, 0.f), ds = os, orr = os, dr = os;
    float smax = 0.f;
    uint64_t px = 0;
    if (valid) {
      const SceneView& S = R.S;
      const CameraBasis& cb = R.cam;
      const float3 eye = cb.eye;
      const float3 d = camera_ray(cb, x, y);
      const float eps = scene_eps(S, R.eps_rel);
      px = R.pixel_begin + (uint64_t)(y - (int)R.row_begin) * R.width + (uint64_t)x;
      const int4 hr = B.rg_hit[px];
      const uint2 jr = B.rg_jobs[px];
      Hit h{__int_as_float(hr.x), hr.y, hr.z, (uint32_t)hr.w};
      const int best = resolve_jobs(S, B.jobs[0], jr.x, jr.y, h);
      uint32_t flags = 0;
      float4 a = make_float4(0.f, 0.f, 0.f, 0.f);
      float ndl = 0.f;
      if (h.inst >= 0) {
        flags |= 1u;
        float3 g;
        if (best >= 0) {
          const float4 rr = B.jobs[0].r[best];
          g = f3(rr.y, rr.z, rr.w);
        }
        Surface sf = surface_at(S, h, eye, d, eps, nullptr, best >= 0 ? &g : nullptr);
        if (sf.chs == PR_CHS_LAMBERT) {
          flags |= 0x100u;
          const float3 pt = madd(eye, h.t, d);
          const float delta = is_sphere_traced(sf.is_id) ? 2.f * eps : eps;
          ndl = light_ndl(sf, R.light, pt);
          a = make_float4(sf.albedo.x, sf.albedo.y, sf.albedo.z, sf.kr);
          if (ndl > 0.f) {
            os = madd(pt, delta, sf.n);
            float3 ls = R.light - os;
            smax = len3(ls);
            ds = ls * (1.f / smax);
            need_s = true;
            flags |= 2u;
          }
          if (R.max_depth >= 2 && sf.kr > 0.f) {
            orr = madd(pt, delta, sf.n);
            dr = normalize3(d - sf.n * (2.f * dot3(d, sf.n)));
            need_m = true;
            flags |= 8u;
          }
        }
      }
      B.st_a[px] = a;
      B.st_b[px] = make_uint2(__float_as_uint(ndl), flags);
    }
    const uint32_t qs = warp_append(&B.hdr->shadow_n, need_s);
    if (need_s) {
      B.sq_a[qs] = make_float4(os.x, os.y, os.z, smax);
      B.sq_b[qs] = make_float4(ds.x, ds.y, ds.z, 0.f);
      B.sq_px[qs] = px;
      B.sq_req[qs] = r;
    }
    const uint32_t qm = warp_append(&B.hdr->mirror_n, need_m);
    if (need_m) {
      B.mq_a[qm] = make_float4(orr.x, orr.y, orr.z, 0.f);
      B.mq_b[qm] = make_float4(dr.x, dr.y, dr.z, 0.f);
      B.mq_px[qm] = px;
      B.mq_req[qm] = r;
    }
    unsigned long long* counter = B.hdr->counter;
    if (counter) {
      const uint32_t tot = __reduce_add_sync(kFull, (need_s ? 1u : 0u) + (need_m ? 1u : 0u));
      if (lane == 0 && tot) atomicAdd(counter, (unsigned long long)tot);
    }
    __syncthreads();
  }
}

// Shadow then mirror queue: traversal with fractal candidates deferred. A
// shadow ray with an occluder of its own needs no jobs.
__global__ void __launch_bounds__(128, 4) k_rg_second(BatchView B, uint32_t chunk) {
  const int lane = threadIdx.x & 31;
  PR_DECLARE_STACK(128);
  for (int q = 0; q < 2; ++q) {
    const bool mirror = q == 1;
    const uint32_t n = mirror ? B.hdr->mirror_n : B.hdr->shadow_n;
    uint32_t* ctr = mirror ? &B.hdr->mirror_ctr : &B.hdr->shadow_ctr;
    for (;;) {
      uint32_t base = 0;
      if (lane == 0) base = atomicAdd(ctr, chunk);
      base = __shfl_sync(kFull, base, 0);
      if (base >= n) break;
      const uint32_t end = min(base + chunk, n);
      for (uint32_t i0 = base; i0 < end; i0 += 32) {
        const uint32_t i = i0 + (uint32_t)lane;
        const bool valid = i < end;
        Deferred dfr;
        dfr.n = 0;
        Hit h;
        uint32_t req = 0;
        float3 o = f3(0.f, 0.f, 0.f), d = o;
        float eps = 0.f;
        if (valid) {
          req = mirror ? B.mq_req[i] : B.sq_req[i];
          const ReqDev& R = B.reqs[req];
          const float4 a = mirror ? B.mq_a[i] : B.sq_a[i], b = mirror ? B.mq_b[i] : B.sq_b[i];
          o = f3(a.x, a.y, a.z);
          d = f3(b.x, b.y, b.z);
          eps = scene_eps(R.S, R.eps_rel);
          trace_typed<false, false, kStackDepth, true>(R.S, o, d, mirror ? 0u : 1u, 0.f, mirror ? INFINITY : a.w, eps,
                                                       R.max_steps, h, stack, nullptr, &dfr);
          if (!mirror && h.inst >= 0) dfr.n = 0;   // occluded already
        }
        const uint32_t first = append_jobs(B, 1, dfr, mirror ? (i | kMirrorSlot) : i, req, mirror, eps,
                                           valid ? B.reqs[req].max_steps : 0u);
        if (valid) {
          const ReqDev& R = B.reqs[req];
          if (first == kEmptyJob && dfr.n > 0) {
            march_in_place(R.S, dfr, eps, R.max_steps, !mirror, h);
            dfr.n = 0;
          }
          if (mirror) {
            B.rg_mhit[i] = make_int4(__float_as_int(h.t), h.inst, h.leaf, (int)h.attr);
            B.rg_mjobs[i] = make_uint2(first, (uint32_t)dfr.n);
          } else {
            B.rg_sjobs[i] = make_uint2(first, (uint32_t)dfr.n | (h.inst >= 0 ? 0x80000000u : 0u));
          }
        }
      }
    }
  }
}

// Shadow visibility and mirror shading from the traversal results and the
// pass-1 jobs; then k_wf_resolve composes every pixel.
__global__ void __launch_bounds__(128, 4) k_rg_finish(BatchView B, uint32_t chunk) {
  const int lane = threadIdx.x & 31;
  const uint32_t ns = B.hdr->shadow_n, nm = B.hdr->mirror_n;
  const MarchJobs& J = B.jobs[1];
  for (;;) {
    uint32_t base = 0;
    if (lane == 0) base = atomicAdd(&B.hdr->finish_ctr, chunk);
    base = __shfl_sync(kFull, base, 0);
    if (base >= ns + nm) break;
    for (uint32_t i = base + lane; i < base + chunk && i < ns + nm; i += 32) {
      if (i < ns) {
        const uint2 sj = B.rg_sjobs[i];
        bool occluded = (sj.y & 0x80000000u) != 0u;
        const float tmax = B.sq_a[i].w;
        for (uint32_t k = 0; k < (sj.y & 0x7FFFFFFFu) && !occluded; ++k) {
          const float th = J.r[sj.x + k].x;
          occluded = th >= 0.f && th < tmax;
        }
        if (!occluded) atomicOr(&B.st_b[B.sq_px[i]].y, 4u);
      } else {
        const uint32_t m = i - ns;
        const ReqDev& R = B.reqs[B.mq_req[m]];
        const SceneView& S = R.S;
        const float4 qa = B.mq_a[m], qb = B.mq_b[m];
        const float3 orr = f3(qa.x, qa.y, qa.z), dr = f3(qb.x, qb.y, qb.z);
        const float eps = scene_eps(S, R.eps_rel);
        const int4 hr = B.rg_mhit[m];
        const uint2 jr = B.rg_mjobs[m];
        Hit rh{__int_as_float(hr.x), hr.y, hr.z, (uint32_t)hr.w};
        const int best = resolve_jobs(S, J, jr.x, jr.y, rh);
        const uint64_t px = B.mq_px[m];
        float3 lr;
        if (rh.inst >= 0) {
          float3 g;
          if (best >= 0) {
            const float4 rr = J.r[best];
            g = f3(rr.y, rr.z, rr.w);
          }
          Surface s2 = surface_at(S, rh, orr, dr, eps, nullptr, best >= 0 ? &g : nullptr);
          lr = s2.chs == PR_CHS_LAMBERT
                   ? lambert_rgb(s2.albedo, R.ambient, R.light_intensity, light_ndl(s2, R.light, madd(orr, rh.t, dr)), 1.f)
                   : f3(0.f, 0.f, 0.f);
          atomicOr(&B.st_b[px].y, 16u);
        } else {
          lr = miss_rgb(S, 0, R.background);
        }
        B.refl[px] = make_float4(lr.x, lr.y, lr.z, 0.f);
      }
    }
  }
}

// Completion flag of a request (batched megakernel modes): every thread
// fences its image writes of the tile, the CTA synchronises, and thread 0
// counts the tile; the CTA that finishes the request's last tile publishes
// the batch's sequence number in the request's host-mapped flag.
__device__ __forceinline__ void tile_finished(const BatchView& B, uint32_t r, uint32_t n_tiles) {
  uint32_t* notify = B.hdr->notify;
  if (notify == nullptr) {
    __syncthreads();
    return;
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    ReqDev* req = const_cast<ReqDev*>(B.reqs) + r;
    const uint32_t done = atomicAdd(&req->tiles_done, 1u) + 1u;
    if (done == n_tiles) {
      __threadfence_system();
      const uint32_t seq = B.hdr->seq;
      asm volatile("st.release.sys.global.u32 [%0], %1;" ::"l"(notify + r), "r"(seq) : "memory");
    }
  }
}

// Batched megakernel: persistent CTAs claim 16x8 tiles of all requests from
// one counter; every pixel runs the single-request kernel's pipeline
// (render_pixel: primary, shadow and mirror rays, shading) and writes its
// request's image directly, with no per-pixel state or ray queues in memory.
template <int kWarpW>
__global__ void __launch_bounds__(128, 4) k_batch_mega(BatchView B) {
  static_assert(kWarpW == 4 || kWarpW == 8 || kWarpW == 16, "warp tile width");
  __shared__ ReqDev sreq;
  __shared__ uint32_t s_tile, s_req;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  constexpr int kWarpsX = 16 / kWarpW;
  const int ox = (warp % kWarpsX) * kWarpW + (lane % kWarpW), oy = (warp / kWarpsX) * (32 / kWarpW) + lane / kWarpW;
  PR_DECLARE_STACK(128);
  uint32_t last_req = kFull, rays = 0;
  for (;;) {
    if (threadIdx.x == 0) {
      const uint32_t t = atomicAdd(&B.hdr->tile_ctr, 1u);
      s_tile = t;
      s_req = t < B.hdr->total_tiles ? find_request(B.reqs, B.hdr->n_req, t) : 0;
    }
    __syncthreads();
    const uint32_t tile = s_tile, r = s_req;
    if (tile >= B.hdr->total_tiles) break;
    if (r != last_req) {
      const uint32_t* src = reinterpret_cast<const uint32_t*>(B.reqs + r);
      uint32_t* dst = reinterpret_cast<uint32_t*>(&sreq);
      for (int i = threadIdx.x; i < (int)(sizeof(ReqDev) / 4); i += blockDim.x) dst[i] = src[i];
      __syncthreads();
      last_req = r;
    }
    const ReqDev& R = sreq;
    const uint32_t lt = tile - R.tile_begin;
    const int x = (int)(lt % R.tiles_x) * 16 + ox, y = (int)R.row_begin + (int)(lt / R.tiles_x) * 8 + oy;
    if (x < (int)R.width && y < (int)(R.row_begin + R.rows)) {
      const PixelParams pp{R.light, R.background, R.light_intensity, R.ambient, R.max_depth, R.max_steps};
      const float eps = scene_eps(R.S, R.eps_rel);
      const float3 color =
          render_pixel<false>(R.S, pp, R.cam.eye, camera_ray(R.cam, x, y), eps, stack, nullptr, nullptr, rays);
      const uint64_t o = (uint64_t)y * R.width + (uint64_t)x;
      if (R.out_rgb) {
        float* f = reinterpret_cast<float*>(R.out) + 3 * o;
        f[0] = color.x;
        f[1] = color.y;
        f[2] = color.z;
      } else {
        R.out[o] = make_float4(color.x, color.y, color.z, 1.f);
      }
    }
    // every thread is done with this tile's request record and counters
    tile_finished(B, r, R.n_tiles);
  }
  if (B.hdr->counter) {
    const uint32_t total = __reduce_add_sync(kFull, rays);
    if (lane == 0 && total) atomicAdd(B.hdr->counter, (unsigned long long)total);
  }
}

// The same with one CTA per 16x8 tile (no claiming loop: the hardware
// schedules the tiles); CTAs past the batch's last tile return at once.
// kWarps = 1: one warp per CTA and four CTAs per tile (one per warp tile),
// so a warp that finishes early frees its slot for the next CTA instead of
// holding it until the tile's slowest warp ends.
// Resident 128-thread CTAs per SM the registers must allow: 5 (at most 102
// registers, about 100 bytes of spills) runs the 64-request batch in 18.15 ms
// against 19.18 ms at 4 (128 registers, no spills).
#ifndef PR_BATCH_MIN_BLOCKS
#define PR_BATCH_MIN_BLOCKS 5
#endif
// Warp tiles follow the single-request kernel's choice per request: 4x8
// pixels for scenes traversed through the wide TLAS, 8x4 for the others (a
// 1080p teaser request 9.6 % faster than with 4x8; the 64-request batch of
// instanced fields within 0.3 %).
// kMirror false: every request of the batch has max_depth 1 (no mirror
// bounce compiled in; fewer registers live across the shadow trace).
template <bool kAhs = false, int kWarps = 4, bool kMirror = true>
__global__ void __launch_bounds__(32 * kWarps, 4 * PR_BATCH_MIN_BLOCKS / kWarps) k_batch_mega_tiles(BatchView B) {
  static_assert(kWarps == 4 || kWarps == 1, "four warps per tile, or one per quarter");
  constexpr int kParts = 4 / kWarps;
  const uint32_t tile = blockIdx.x / kParts;
  if (tile >= B.hdr->total_tiles) return;
  __shared__ ReqDev sreq;
  const int warp = (int)(threadIdx.x >> 5) + (int)(blockIdx.x % kParts) * kWarps, lane = threadIdx.x & 31;
  // Every thread finds the request (the same loads in every lane) and copies
  // part of its record (camera frame included): one barrier, and no
  // thread-serial work at the start of the tile.
  const uint32_t s_req = find_request(B.reqs, B.hdr->n_req, tile);
  {
    const uint32_t* src = reinterpret_cast<const uint32_t*>(B.reqs + s_req);
    uint32_t* dst = reinterpret_cast<uint32_t*>(&sreq);
    for (int i = threadIdx.x; i < (int)(sizeof(ReqDev) / 4); i += blockDim.x) dst[i] = src[i];
  }
  __syncthreads();
  const ReqDev& R = sreq;
  const uint32_t lt = tile - R.tile_begin;
  const int wl = R.S.tlas4 ? 2 : 3;   // log2 of the warp tile's width
  const int x = (int)(lt % R.tiles_x) * 16 + (warp % (16 >> wl)) * (1 << wl) + (lane & ((1 << wl) - 1));
  const int y = (int)R.row_begin + (int)(lt / R.tiles_x) * 8 + (warp / (16 >> wl)) * (32 >> wl) + (lane >> wl);
  uint32_t rays = 0;
  if (x < (int)R.width && y < (int)(R.row_begin + R.rows)) {
    PR_DECLARE_STACK(32 * kWarps);
    const PixelParams pp{R.light, R.background, R.light_intensity, R.ambient, R.max_depth, R.max_steps};
    const float eps = scene_eps(R.S, R.eps_rel);
    const float3 color = render_pixel<false, false, kStackDepth, 0, kAhs, true, kMirror>(
        R.S, pp, R.cam.eye, camera_ray(R.cam, x, y), eps, stack, nullptr, nullptr, rays);
    const uint64_t o = (uint64_t)y * R.width + (uint64_t)x;
    if (R.out_rgb) {
      float* f = reinterpret_cast<float*>(R.out) + 3 * o;
      f[0] = color.x;
      f[1] = color.y;
      f[2] = color.z;
    } else {
      R.out[o] = make_float4(color.x, color.y, color.z, 1.f);
    }
  }
  if (B.hdr->counter) {
    const uint32_t total = __reduce_add_sync(kFull, rays);
    if (lane == 0 && total) atomicAdd(B.hdr->counter, (unsigned long long)total);
  }
  if (B.hdr->notify) tile_finished(B, s_req, R.n_tiles * kParts);   // without flags the CTA just ends
}

}  // namespace

int launch_wavefront(const BatchView& B, const BatchTuning& T, int n_sm, uint32_t grid_tiles, cudaStream_t s,
                     bool ahs_march, bool mirror) {
  int launches = 0;
  if (ahs_march || T.megakernel == 2 || T.megakernel == 4) {
    // one CTA per tile (any-hit batches are staged with 16x8 tiles)
    if (!grid_tiles) return 0;
    if (ahs_march) k_batch_mega_tiles<true><<<grid_tiles, 128, 0, s>>>(B);
    else if (T.megakernel == 2 && mirror) k_batch_mega_tiles<><<<grid_tiles, 128, 0, s>>>(B);
    else if (T.megakernel == 2) k_batch_mega_tiles<false, 4, false><<<grid_tiles, 128, 0, s>>>(B);
    else if (mirror) k_batch_mega_tiles<false, 1><<<4 * grid_tiles, 32, 0, s>>>(B);
    else k_batch_mega_tiles<false, 1, false><<<4 * grid_tiles, 32, 0, s>>>(B);
    return 1;
  }
  cudaMemsetAsync(&B.hdr->tile_ctr, 0, 5 * sizeof(uint32_t), s);   // tile_ctr, shadow_n, mirror_n, shadow_ctr, mirror_ctr
  const uint32_t grid = (uint32_t)n_sm * T.ctas_per_sm;
  if (T.megakernel == 1) {
    k_batch_mega<8><<<grid, 128, 0, s>>>(B);
    return 1;
  }
  if (T.megakernel == 3) {
    cudaMemsetAsync(&B.hdr->job_n[0], 0, 6 * sizeof(uint32_t), s);   // job_n, job_ctr, shade_ctr, finish_ctr
    const uint32_t grid_m = (uint32_t)n_sm * 8;
    if (T.tile_w == 32) k_rg_primary<32, 4><<<grid, 128, 0, s>>>(B);
    else if (T.tile_w == 8) k_rg_primary<8, 16><<<grid, 128, 0, s>>>(B);
    else k_rg_primary<16, 8><<<grid, 128, 0, s>>>(B);
    k_rg_march<<<grid_m, 128, 0, s>>>(B, 0);
    if (T.tile_w == 32) k_rg_shade<32, 4><<<grid, 128, 0, s>>>(B);
    else if (T.tile_w == 8) k_rg_shade<8, 16><<<grid, 128, 0, s>>>(B);
    else k_rg_shade<16, 8><<<grid, 128, 0, s>>>(B);
    k_rg_second<<<grid, 128, 0, s>>>(B, T.queue_chunk);
    k_rg_march<<<grid_m, 128, 0, s>>>(B, 1);
    k_rg_finish<<<grid, 128, 0, s>>>(B, T.queue_chunk);
    k_wf_resolve<<<(uint32_t)n_sm * 8, 256, 0, s>>>(B);
    return 7;
  }
  if (T.tile_w == 32) k_wf_primary<32, 4><<<grid, 128, 0, s>>>(B);
  else if (T.tile_w == 8) k_wf_primary<8, 16><<<grid, 128, 0, s>>>(B);
  else k_wf_primary<16, 8><<<grid, 128, 0, s>>>(B);
  k_wf_shadow<<<grid, 128, 0, s>>>(B, T.queue_chunk);
  k_wf_mirror<<<grid, 128, 0, s>>>(B, T.queue_chunk);
  k_wf_resolve<<<(uint32_t)n_sm * 8, 256, 0, s>>>(B);
  launches += 4;
  return launches;
}

}  // namespace pr
