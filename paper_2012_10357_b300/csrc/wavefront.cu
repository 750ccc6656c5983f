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
  __shared__ CameraBasis scam;
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
      if (threadIdx.x == 0) scam = camera_basis(sreq.cam, sreq.width, sreq.height);
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
      const float3 eye = scam.eye;
      const float3 d = camera_ray(scam, x, y);
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
  __shared__ CameraBasis scam;
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
      if (threadIdx.x == 0) scam = camera_basis(sreq.cam, sreq.width, sreq.height);
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
          render_pixel<false>(R.S, pp, scam.eye, camera_ray(scam, x, y), eps, stack, nullptr, nullptr, rays);
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
template <int kWarpW>
__global__ void __launch_bounds__(128, 4) k_batch_mega_tiles(BatchView B) {
  const uint32_t tile = blockIdx.x;
  if (tile >= B.hdr->total_tiles) return;
  __shared__ ReqDev sreq;
  __shared__ CameraBasis scam;
  __shared__ uint32_t s_req;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  constexpr int kWarpsX = 16 / kWarpW;
  if (threadIdx.x == 0) s_req = find_request(B.reqs, B.hdr->n_req, tile);
  __syncthreads();
  {
    const uint32_t* src = reinterpret_cast<const uint32_t*>(B.reqs + s_req);
    uint32_t* dst = reinterpret_cast<uint32_t*>(&sreq);
    for (int i = threadIdx.x; i < (int)(sizeof(ReqDev) / 4); i += blockDim.x) dst[i] = src[i];
  }
  __syncthreads();
  if (threadIdx.x == 0) scam = camera_basis(sreq.cam, sreq.width, sreq.height);
  __syncthreads();
  const ReqDev& R = sreq;
  const uint32_t lt = tile - R.tile_begin;
  const int x = (int)(lt % R.tiles_x) * 16 + (warp % kWarpsX) * kWarpW + (lane % kWarpW);
  const int y = (int)R.row_begin + (int)(lt / R.tiles_x) * 8 + (warp / kWarpsX) * (32 / kWarpW) + lane / kWarpW;
  uint32_t rays = 0;
  if (x < (int)R.width && y < (int)(R.row_begin + R.rows)) {
    PR_DECLARE_STACK(128);
    const PixelParams pp{R.light, R.background, R.light_intensity, R.ambient, R.max_depth, R.max_steps};
    const float eps = scene_eps(R.S, R.eps_rel);
    const float3 color = render_pixel<false>(R.S, pp, scam.eye, camera_ray(scam, x, y), eps, stack, nullptr, nullptr, rays);
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
  tile_finished(B, s_req, R.n_tiles);
}

}  // namespace

int launch_wavefront(const BatchView& B, const BatchTuning& T, int n_sm, uint32_t grid_tiles, cudaStream_t s) {
  int launches = 0;
  if (T.megakernel == 2) {
    if (grid_tiles) k_batch_mega_tiles<8><<<grid_tiles, 128, 0, s>>>(B);
    return grid_tiles ? 1 : 0;
  }
  cudaMemsetAsync(&B.hdr->tile_ctr, 0, 5 * sizeof(uint32_t), s);   // tile_ctr, shadow_n, mirror_n, shadow_ctr, mirror_ctr
  const uint32_t grid = (uint32_t)n_sm * T.ctas_per_sm;
  if (T.megakernel == 1) {
    k_batch_mega<8><<<grid, 128, 0, s>>>(B);
    return 1;
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
