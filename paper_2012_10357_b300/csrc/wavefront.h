// Device-side layout of the batched wavefront path.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "pr_device.cuh"

namespace pr {

// One request as the kernels see it (copied to shared memory per tile).
struct ReqDev {
  SceneView S;
  CameraBasis cam;                   // camera frame of the image (camera_frame on the host)
  float3 light, background;
  float light_intensity, eps_rel, ambient;
  uint32_t width, height, max_depth, max_steps;
  uint32_t row_begin, rows;          // rendered rows [row_begin, row_begin + rows) of the image
  uint32_t tile_begin, tiles_x;
  float4* out;                       // float4 per pixel, or 3 floats with out_rgb
  uint64_t pixel_begin;
  uint32_t out_rgb, n_tiles;         // n_tiles: tiles of this request in the batch
  uint32_t tiles_done, pad_[3];      // tiles finished (megakernel modes with completion flags)
};

// Counters and totals of the current batch (device memory).
struct BatchHdr {
  uint32_t n_req, total_tiles;
  uint64_t total_pixels;
  uint32_t tile_ctr, shadow_n, mirror_n, shadow_ctr, mirror_ctr, pad;
  unsigned long long* counter;   // rays traced (optional)
  // Completion flags (optional, megakernel modes): when the last tile of
  // request r is written, notify[r] = seq. notify is host-mapped memory.
  uint32_t* notify;
  uint32_t seq, pad2;
  // regrouped mode: march jobs appended / claimed per pass (0 primary, 1 shadow + mirror)
  uint32_t job_n[2], job_ctr[2];
  uint32_t shade_ctr, finish_ctr, pad3[2];
};

// One deferred fractal march (regrouped mode), self-contained so that a lane
// starting a job issues independent loads only (128 bytes):
//   a[0] = object-space origin xyz, t_lo    a[1] = object-space direction xyz, t_hi
//   a[2] = instance, leaf, shader id | normal << 16, ray slot (bits)
//   a[3] = eps, step cap (bits), request (bits), unused
//   a[4..6] = the primitive's first three parameter rows
//   r = (t or -1 for a miss, gradient xyz), written by the march kernel
constexpr int kJobRows = 7;
struct MarchJobs {
  float4* a;   // [cap][kJobRows]
  float4* r;   // [cap]
};

struct BatchView {
  BatchHdr* hdr;
  const ReqDev* reqs;
  float4* st_a;       // [pixels] albedo rgb, reflectance
  uint2* st_b;        // [pixels] n.l bits, flags
  float4* refl;       // [pixels] mirror radiance
  float4 *sq_a, *sq_b;  // shadow queue: origin+tmax, direction
  uint64_t* sq_px;
  uint32_t* sq_req;
  float4 *mq_a, *mq_b;  // mirror queue
  uint64_t* mq_px;
  uint32_t* mq_req;
  // regrouped mode: traversal results per ray slot (primary: pixel; shadow /
  // mirror: queue position) and the deferred march jobs of each pass
  int4* rg_hit;       // [pixels] primary ray: closest non-fractal hit (t bits, instance, leaf, attr)
  uint2* rg_jobs;     // [pixels] primary ray: first job, job count
  int4* rg_mhit;      // [mirror slots] mirror ray hit
  uint2* rg_mjobs;    // [mirror slots] mirror ray jobs
  uint2* rg_sjobs;    // [shadow slots] shadow ray: first job, job count | occluded << 31
  MarchJobs jobs[2];  // pass 0 (primary) and pass 1 (shadow and mirror)
  uint32_t job_cap;   // jobs per pass
  uint32_t max_req;
};

struct BatchTuning {
  uint32_t ctas_per_sm, tile_w, tile_h, queue_chunk;
  // 1: one persistent megakernel (16x8 tiles), 2: one CTA per 16x8 tile, 0: four
  // stages, 3: regrouped stages (fractal marches deferred into a job queue),
  // 4: one one-warp CTA per 4x8 quarter of each 16x8 tile
  uint32_t megakernel;
};

// grid_tiles: tiles the one-CTA-per-tile megakernels launch for (at least the batch's tiles); unused otherwise
// ahs_march: a request's scene has an any-hit shader on a sphere-traced shader;
// the batch then runs the one-CTA-per-tile megakernel compiled with the
// any-hit march (staged with 16x8 tiles), whatever T says.
// mirror: a request has max_depth 2; when none has, the one-CTA-per-tile
// megakernels run a variant without the mirror bounce.
int launch_wavefront(const BatchView& B, const BatchTuning& T, int n_sm, uint32_t grid_tiles, cudaStream_t s,
                     bool ahs_march = false, bool mirror = true);

}  // namespace pr
