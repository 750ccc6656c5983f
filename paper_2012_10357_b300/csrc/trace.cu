// Megakernel tracer: one thread per pixel runs the whole per-pixel pipeline
// the paper sets up through DXR (Section 2.2.3): ray generation, TLAS/BLAS
// traversal in software, Eq. 1 shader-table dispatch to the hit group's
// intersection shader, closest-hit shading with a shadow ray (and one mirror
// ray), miss shaders, and the framebuffer write.
#include <cuda_runtime.h>

#include <cstdint>

#include "internal.h"
#include "shaders.cuh"
#include "tracer.cuh"

namespace pr {
namespace {

struct Params {
  SceneView S;
  pr_camera cam0;
  const pr_camera* cams;
  uint32_t width, height, max_depth, max_steps, flags;
  float3 light, background;
  float light_intensity, eps_rel, ambient;
  float4* out;
  pr_aov* aov;
  unsigned long long* counter;
};

// Resident CTAs per SM the register allocation must allow (occupancy knob;
// 4 x 128 threads -> at most 128 registers, 4 x 32 KB shared stacks).
#ifndef PR_TRACE_MIN_BLOCKS
#define PR_TRACE_MIN_BLOCKS 4
#endif
// Width of a warp's pixel tile (height 32 / width). Measured on B300: 8x4 is
// best for scenes of few instances (the teaser: 8x4 13.1, 4x8 11.6, 16x2 12.6
// Grays/s), 4x8 for large instanced fields (+2 % at 100 000 instances). The
// launch picks 4x8 for scenes traversed through the 4-wide TLAS.
#ifndef PR_WARP_TILE_W
#define PR_WARP_TILE_W 8
#endif
#ifndef PR_WARP_TILE_W_WIDE
#define PR_WARP_TILE_W_WIDE 4
#endif

template <bool kStats, int kWarpW>
__global__ void __launch_bounds__(128, PR_TRACE_MIN_BLOCKS) k_trace(Params P, unsigned long long* work) {
  static_assert(kWarpW == 4 || kWarpW == 8 || kWarpW == 16, "warp tile width");
  const SceneView& S = P.S;
  WorkCounters wcl;
  if (kStats) memset(&wcl, 0, sizeof(wcl));
  WorkCounters* wc = kStats ? &wcl : nullptr;
  const uint32_t frame = blockIdx.z;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // 16x8-pixel CTA tile split into four warp tiles of kWarpW x (32 / kWarpW) pixels
  constexpr int kWarpsX = 16 / kWarpW;
  const int x = blockIdx.x * 16 + (warp % kWarpsX) * kWarpW + (lane % kWarpW);
  const int y = blockIdx.y * 8 + (warp / kWarpsX) * (32 / kWarpW) + lane / kWarpW;
  const bool valid = x < (int)P.width && y < (int)P.height;
  __shared__ CameraBasis s_cam;
  if (threadIdx.x == 0) s_cam = camera_basis(P.cams ? P.cams[frame] : P.cam0, P.width, P.height);
  __syncthreads();
  uint32_t rays = 0;
  if (valid) {
    PR_DECLARE_STACK(128);
    const float3 eye = s_cam.eye;
    const float3 d = camera_ray(s_cam, x, y);
    const float eps = scene_eps(S, P.eps_rel);

    Hit h;
    rays = 1;
    trace_typed<kStats>(S, eye, d, 0, 0.f, INFINITY, eps, P.max_steps, h, stack, wc);
    const size_t pix = ((size_t)frame * P.height + (size_t)y) * P.width + (size_t)x;
    // AOV fields are stored as soon as they are known, so none of them stays
    // live across the shadow and mirror traces
    pr_aov* av = P.aov ? P.aov + pix : nullptr;
    float3 color;
    uint32_t flags = 0;
    if (h.inst < 0) {
      color = miss_rgb(S, 0, P.background);
      if (av) {
        av->t = -1.f;
        av->inst = av->geom = av->prim = PR_NONE;
        av->n[0] = av->n[1] = av->n[2] = 0.f;
      }
    } else {
      flags |= 1u;
      Surface sf = surface_at(S, h, eye, d, eps, wc);
      if (av) {
        av->t = h.t;
        av->inst = (uint32_t)h.inst;
        av->geom = sf.geom;
        av->prim = sf.prim;
        av->n[0] = sf.n.x; av->n[1] = sf.n.y; av->n[2] = sf.n.z;
      }
      if (sf.chs != PR_CHS_LAMBERT) {
        color = f3(0.f, 0.f, 0.f);
      } else {
        const float3 pt = madd(eye, h.t, d);
        const float delta = is_sphere_traced(sf.is_id) ? 2.f * eps : eps;
        const float ndl = light_ndl(sf, P.light, pt);
        float vis = 1.f;
        if (ndl > 0.f) {
          // shadow ray: offset origin, toward the light, ends at the light
          float3 os = madd(pt, delta, sf.n);
          float3 ls = P.light - os;
          float dist = len3(ls);
          Hit sh;
          rays++;
          flags |= 2u;
          trace_typed<kStats>(S, os, ls * (1.f / dist), 1, 0.f, dist, eps, P.max_steps, sh, stack, wc);
          vis = sh.inst >= 0 ? 0.f : 1.f;
          if (sh.inst < 0) flags |= 4u;
        }
        color = lambert_rgb(sf.albedo, P.ambient, P.light_intensity, ndl, vis);
        if (P.max_depth >= 2 && sf.kr > 0.f) {
          // one mirror bounce, its hit shaded without a shadow ray
          float3 orr = madd(pt, delta, sf.n);
          float3 dr = normalize3(d - sf.n * (2.f * dot3(d, sf.n)));
          const float kr = sf.kr;
          Hit rh;
          rays++;
          flags |= 8u;
          trace_typed<kStats>(S, orr, dr, 0, 0.f, INFINITY, eps, P.max_steps, rh, stack, wc);
          float3 lr;
          if (rh.inst >= 0) {
            flags |= 16u;
            Surface s2 = surface_at(S, rh, orr, dr, eps, wc);
            if (av) {
              av->refl_t = rh.t;
              av->refl_inst = (uint32_t)rh.inst;
              av->refl_geom = s2.geom;
              av->refl_prim = s2.prim;
            }
            lr = s2.chs == PR_CHS_LAMBERT
                     ? lambert_rgb(s2.albedo, P.ambient, P.light_intensity, light_ndl(s2, P.light, madd(orr, rh.t, dr)), 1.f)
                     : f3(0.f, 0.f, 0.f);
          } else {
            lr = miss_rgb(S, 0, P.background);
          }
          color = mirror_mix(color, lr, kr);
        }
      }
    }
    if (P.flags & PR_TRACE_OUTPUT_RGB) {
      float* o = reinterpret_cast<float*>(P.out) + 3 * pix;
      o[0] = color.x;
      o[1] = color.y;
      o[2] = color.z;
    } else {
      P.out[pix] = make_float4(color.x, color.y, color.z, 1.f);
    }
    if (av) {
      if (!(flags & 16u)) {
        av->refl_t = -1.f;
        av->refl_inst = av->refl_geom = av->refl_prim = PR_NONE;
      }
      av->flags = flags;
    }
  }
  if (P.counter) {
    uint32_t total = __reduce_add_sync(0xFFFFFFFFu, rays);
    if (lane == 0 && total) atomicAdd(P.counter, (unsigned long long)total);
  }
  if (kStats) {
    const uint32_t* c = reinterpret_cast<const uint32_t*>(&wcl);
    for (int i = 0; i < (int)(sizeof(WorkCounters) / 4); ++i) {
      uint32_t v = __reduce_add_sync(0xFFFFFFFFu, c[i]);
      if (lane == 0 && v) atomicAdd(work + i, (unsigned long long)v);
    }
  }
}

}  // namespace

int launch_trace(const TraceLaunch& L, cudaStream_t s) {
  Params P;
  P.S = L.S;
  P.cam0 = L.cam0;
  P.cams = L.cams;
  P.width = L.width;
  P.height = L.height;
  P.max_depth = L.max_depth;
  P.max_steps = L.max_steps;
  P.flags = L.flags;
  P.light = make_float3(L.light[0], L.light[1], L.light[2]);
  P.background = make_float3(L.background[0], L.background[1], L.background[2]);
  P.light_intensity = L.light_intensity;
  P.eps_rel = L.eps_rel;
  P.ambient = L.ambient;
  P.out = L.out;
  P.aov = (L.flags & PR_TRACE_WRITE_AOV) ? L.aov : nullptr;
  P.counter = L.counter;
  dim3 grid((L.width + 15) / 16, (L.height + 7) / 8, L.n_frames);
  if (L.S.tlas4) {
    if (L.work) k_trace<true, PR_WARP_TILE_W_WIDE><<<grid, 128, 0, s>>>(P, L.work);
    else k_trace<false, PR_WARP_TILE_W_WIDE><<<grid, 128, 0, s>>>(P, nullptr);
  } else {
    if (L.work) k_trace<true, PR_WARP_TILE_W><<<grid, 128, 0, s>>>(P, L.work);
    else k_trace<false, PR_WARP_TILE_W><<<grid, 128, 0, s>>>(P, nullptr);
  }
  return 1;
}

}  // namespace pr
