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
  CameraBasis cam0;            // the frame of a one-frame launch (kernel parameter space)
  const CameraBasis* cams;     // frames of a multi-frame launch (device), or null
  uint32_t width, height, flags;
  float eps_rel;
  PixelParams px;
  float4* out;
  pr_aov* aov;
  unsigned long long* counter;
};

// Resident CTAs per SM the register allocation must allow (occupancy knob;
// 4 x 128 threads -> at most 128 registers, 4 x 32 KB shared stacks; 5 -> at
// most 102 registers, a few spills). Scenes traversed through the wide TLAS
// (instanced fields) take 5 (100 000-instance field at 3840x2160: 2.20 -> 2.33
// Grays/s), scenes of few instances 4 (the teaser: 0.5 % faster than at 5).
#ifndef PR_TRACE_MIN_BLOCKS
#define PR_TRACE_MIN_BLOCKS 4
#endif
#ifndef PR_TRACE_MIN_BLOCKS_WIDE
#define PR_TRACE_MIN_BLOCKS_WIDE 5
#endif
// Variants without the mirror bounce (launches with max_depth 1: the
// instanced field, batch requests): the shadow trace is the last, so fewer
// registers are live across it and the register bound for 5 CTAs/SM (96
// registers) leaves no spills. Measured on B300 (100 000-instance field at
// 3840x2160, build + frame): 2 369 -> 2 460 Mrays/s against the
// mirror-capable kernel; 6 CTAs/SM (80 registers, 104 bytes of spills) 2 348.
#ifndef PR_TRACE_MIN_BLOCKS_WIDE1
#define PR_TRACE_MIN_BLOCKS_WIDE1 5
#endif
#ifndef PR_TRACE_MIN_BLOCKS1
#define PR_TRACE_MIN_BLOCKS1 5
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

// kAnalytic: scenes without sphere-traced shaders whose stack bound fits the
// short stack (kShortStackDepth entries, 4 KB per CTA instead of 32 KB); the
// estimator code is not compiled in, so the kernel fits 102 registers and 5
// CTAs stay resident instead of 4. Same arithmetic, same bits. Measured on
// B300 (4096 jittered 64x64 frames of the small analytic scene per launch,
// traversal inline at one site): 33.9 / 38.6 / 36.7 Grays/s at 4 / 5 / 6
// CTAs per SM (106 registers without spills; 92 and 256 bytes of spill loads).
#ifndef PR_TRACE_MIN_BLOCKS_ANALYTIC
#define PR_TRACE_MIN_BLOCKS_ANALYTIC 5
#endif
// The analytic variant without the mirror bounce (config-1 frames), and its
// copy for launches without an AOV buffer (kAov false): 4096 frames on B300,
// 39.3 Grays/s with the mirror-capable kernel; without the bounce 40.9 /
// 42.0 / 40.9 / 41.8 Grays/s at 5 / 6 / 7 / 8 CTAs/SM; with no AOV code
// either (and the primary ray's surface read from the loop's ray, so the
// camera ray is not kept live) 44.4 / 44.2 / 45.1 Grays/s at 6 / 7 / 8 CTAs/SM
// (80 / 72 / 64 registers, 56 / 112 / 196 bytes of spills: the extra warps
// hide more latency than the spills cost).
#ifndef PR_TRACE_MIN_BLOCKS_ANALYTIC1
#define PR_TRACE_MIN_BLOCKS_ANALYTIC1 8
#endif

// kAov false: the launch writes no AOV buffer (no AOV stores compiled in).
template <bool kStats, int kWarpW, bool kAnalytic, int kTlas = 0, bool kAhs = false, bool kMirror = true,
          bool kAov = true>
__global__ void __launch_bounds__(128, kAnalytic && !kMirror            ? PR_TRACE_MIN_BLOCKS_ANALYTIC1
                                      : kAnalytic                       ? PR_TRACE_MIN_BLOCKS_ANALYTIC
                                      : kWarpW == PR_WARP_TILE_W_WIDE && !kMirror ? PR_TRACE_MIN_BLOCKS_WIDE1
                                      : kWarpW == PR_WARP_TILE_W_WIDE ? PR_TRACE_MIN_BLOCKS_WIDE
                                      : !kMirror                      ? PR_TRACE_MIN_BLOCKS1
                                                                      : PR_TRACE_MIN_BLOCKS)
    k_trace(Params P, unsigned long long* work) {
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
  uint32_t rays = 0;
  if (valid) {
    PR_DECLARE_STACK_N(128, kAnalytic ? kShortStackDepth : kStackDepth);
    // the frame comes from the host (parameter space, or the frames' array): no set-up per CTA
    const CameraBasis cb = P.cams ? P.cams[frame] : P.cam0;
    const float3 eye = cb.eye;
    const float3 d = camera_ray(cb, x, y);
    const float eps = scene_eps(S, P.eps_rel);

    const size_t pix = ((size_t)frame * P.height + (size_t)y) * P.width + (size_t)x;
    const float3 color = render_pixel<kStats, kAnalytic, kAnalytic ? kShortStackDepth : kStackDepth, kTlas, kAhs, true, kMirror>(
        S, P.px, eye, d, eps, stack, wc, kAov && P.aov ? P.aov + pix : nullptr, rays);
    if (P.flags & PR_TRACE_OUTPUT_RGB) {
      float* o = reinterpret_cast<float*>(P.out) + 3 * pix;
      o[0] = color.x;
      o[1] = color.y;
      o[2] = color.z;
    } else {
      P.out[pix] = make_float4(color.x, color.y, color.z, 1.f);
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
  P.flags = L.flags;
  P.eps_rel = L.eps_rel;
  P.px.max_depth = L.max_depth;
  P.px.max_steps = L.max_steps;
  P.px.light = make_float3(L.light[0], L.light[1], L.light[2]);
  P.px.background = make_float3(L.background[0], L.background[1], L.background[2]);
  P.px.light_intensity = L.light_intensity;
  P.px.ambient = L.ambient;
  P.out = L.out;
  P.aov = (L.flags & PR_TRACE_WRITE_AOV) ? L.aov : nullptr;
  P.counter = L.counter;
  dim3 grid((L.width + 15) / 16, (L.height + 7) / 8, L.n_frames);
  // kernel variant: TLAS form x stats x any-hit march (analytic scenes never need the latter)
  auto go = [&](auto kernel) { kernel<<<grid, 128, 0, s>>>(P, L.work); };
  const bool st = L.work != nullptr;
  if (L.S.tlas8 && L.S.tlas8_format == kWide8Q) {
    if (L.ahs_march) st ? go(k_trace<true, PR_WARP_TILE_W_WIDE, false, kWide8Q, true>)
                        : go(k_trace<false, PR_WARP_TILE_W_WIDE, false, kWide8Q, true>);
    else st ? go(k_trace<true, PR_WARP_TILE_W_WIDE, false, kWide8Q>) : go(k_trace<false, PR_WARP_TILE_W_WIDE, false, kWide8Q>);
  } else if (L.S.tlas8) {
    if (L.ahs_march) st ? go(k_trace<true, PR_WARP_TILE_W_WIDE, false, kWide8, true>)
                        : go(k_trace<false, PR_WARP_TILE_W_WIDE, false, kWide8, true>);
    else st ? go(k_trace<true, PR_WARP_TILE_W_WIDE, false, kWide8>) : go(k_trace<false, PR_WARP_TILE_W_WIDE, false, kWide8>);
  } else if (L.S.tlas4) {
    if (L.ahs_march) st ? go(k_trace<true, PR_WARP_TILE_W_WIDE, false, 0, true>)
                        : go(k_trace<false, PR_WARP_TILE_W_WIDE, false, 0, true>);
    else if (L.max_depth < 2) st ? go(k_trace<true, PR_WARP_TILE_W_WIDE, false, 0, false, false>)
                                 : go(k_trace<false, PR_WARP_TILE_W_WIDE, false, 0, false, false>);
    else st ? go(k_trace<true, PR_WARP_TILE_W_WIDE, false>) : go(k_trace<false, PR_WARP_TILE_W_WIDE, false>);
  } else if (L.analytic_small) {
    if (L.max_depth >= 2) st ? go(k_trace<true, PR_WARP_TILE_W, true>) : go(k_trace<false, PR_WARP_TILE_W, true>);
    else if (P.aov) st ? go(k_trace<true, PR_WARP_TILE_W, true, 0, false, false>) : go(k_trace<false, PR_WARP_TILE_W, true, 0, false, false>);
    else st ? go(k_trace<true, PR_WARP_TILE_W, true, 0, false, false, false>)
            : go(k_trace<false, PR_WARP_TILE_W, true, 0, false, false, false>);
  } else {
    if (L.ahs_march) st ? go(k_trace<true, PR_WARP_TILE_W, false, 0, true>) : go(k_trace<false, PR_WARP_TILE_W, false, 0, true>);
    else if (L.max_depth < 2) st ? go(k_trace<true, PR_WARP_TILE_W, false, 0, false, false>)
                                 : go(k_trace<false, PR_WARP_TILE_W, false, 0, false, false>);
    else st ? go(k_trace<true, PR_WARP_TILE_W, false>) : go(k_trace<false, PR_WARP_TILE_W, false>);
  }
  return 1;
}

}  // namespace pr
