// Host-side internals shared by the C ABI, the BVH builder and the tracer.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "pr_device.cuh"

namespace pr {

// One BVH level to build: leaves are boxes[gather ? gather[k] : k] (6 floats),
// k = 0..n-1 in input order; a leaf ref is kLeafBit | (leaf_ref_base + k).
struct LevelDesc {
  const float* boxes;
  const uint32_t* gather;
  uint32_t n;
  uint32_t leaf_ref_base;
  float4* nodes;       // [n-1][4]
  uint32_t* perm;      // [n] sorted position -> k
  uint32_t* codes;     // [n] Morton code by sorted position
  float* root_box;     // 8 floats: lo.xyz, 0, hi.xyz, 0
};

// Scratch of the multi-kernel (large level) path.
struct BuildScratch {
  uint32_t* keys[2];
  uint32_t* vals[2];
  uint32_t* hist;        // [256 * max_tiles]
  uint32_t* counters;    // [max_n]
  uint32_t* parent_int;  // [max_n]
  uint32_t* parent_leaf; // [max_n]
  float* partial;        // [kMaxPartials * 6]
  float* cluster_boxes;  // [2 * max_n * 8] PLOC cluster records (may alias a buffer free during the build)
  uint32_t max_n;
};

constexpr uint32_t kSmallMax = 1024;      // levels up to this size build in one CTA
constexpr uint32_t kSortTile = 2048;      // keys per tile in the radix sort
constexpr uint32_t kMaxPartials = 1024;   // blocks of the centroid-bounds pass

inline uint32_t sort_tiles(uint32_t n) { return (n + kSortTile - 1) / kSortTile; }

// Launchers (bvh.cu). Each returns the number of kernels launched.
int launch_build_small(const LevelDesc* d_jobs, uint32_t n_jobs, cudaStream_t s);
int launch_build_small_one(const LevelDesc& job, cudaStream_t s);
// 4-wide collapse of a built binary level of n leaves (scratch: parent, even, rank of n words).
int launch_collapse4(const float4* nodes2, uint32_t n, uint32_t* parent, uint32_t* even, uint32_t* rank,
                     float4* nodes4, cudaStream_t s);

// Greedy collapse of a binary tree (root 0, n leaves) into wide nodes: each
// wide node opens its largest-area internal child until it has W children.
// Formats: kWide4 (128-B 4-wide nodes, the layout of launch_collapse4),
// kWide8 (224-B float 8-wide), kWide8Q (96-B quantised 8-wide).
struct WideScratch {
  uint32_t* slots;       // [8 * (n - 1)] child slots per binary node
  uint32_t* is_root;     // [n] binary node roots a wide node
  uint32_t* rank;        // [n] wide node index (exclusive prefix sum of is_root)
  uint32_t* frontier;    // [n] roots handed from the top-down pass to the per-root pass
  uint32_t* n_frontier;  // [1]
};
int launch_collapse_wide(const float4* nodes2, uint32_t n, int format, const WideScratch& ws, float4* out,
                         uint32_t* error_word, cudaStream_t s);
int launch_build_large(const LevelDesc& job, const BuildScratch& sc, cudaStream_t s);

// PLOC build of a large level (more than kSmallMax leaves): the LBVH's Morton
// sort, then bottom-up clustering in one cooperative launch, same node layout;
// needs sc.cluster_boxes (16 floats per leaf). The clustering launch waits for
// `after` and records `mark` (each optional): pr_build_bvh_many_ex orders the
// clustering launches of concurrent builds one after another with them.
// Returns the launches issued, or -1 when a launch was refused.
struct PlocArgs {
  LevelDesc J;
  const uint32_t* codes;     // sorted Morton codes
  const uint32_t* vals;      // leaves in Morton order
  float4* R[2];              // cluster records [m][2] (lo.xyz + ref bits, hi.xyz), double-buffered
  int* nn;                   // nearest neighbour of each cluster
  unsigned long long* part;  // per-block (survivors | merges << 32)
  uint32_t* hdr;             // done, abort, barrier count, barrier generation
  uint32_t* error_word;      // gets 1 << PR_ERR_TIMEOUT when a barrier gives up (optional)
};
int launch_build_ploc(const LevelDesc& job, const BuildScratch& sc, uint32_t* error_word, cudaStream_t s,
                      cudaEvent_t after = nullptr, cudaEvent_t mark = nullptr);

// Scratch bytes of the large-level path for n leaves, and its carving.
size_t build_scratch_bytes(uint32_t n);
BuildScratch carve_build_scratch(void* base, uint32_t n);
int launch_triangle_boxes(const float* vertices, const uint32_t* indices, uint32_t n_tri, float* boxes,
                          cudaStream_t s);
// Inputs and outputs of the instance pass (world boxes, records).
struct InstanceArgs {
  const float* xform;
  const uint32_t *inst_blas, *inst_id, *inst_sbt, *inst_mask;
  const float4* blas_box;
  const int4* blas_info;
  uint32_t n;
  float* boxes;
  float4* rec;
};
int launch_instances(const InstanceArgs& A, cudaStream_t s);
// BLAS levels, instances and TLAS of a small scene in one single-CTA launch;
// d_jobs holds the n_blas_jobs BLAS levels followed by the TLAS level.
int launch_build_scene_small(const LevelDesc* d_jobs, uint32_t n_blas_jobs, const InstanceArgs& A, cudaStream_t s);

// Tracer (trace.cu).
struct TraceLaunch {
  SceneView S;
  CameraBasis cam0;            // frame of a one-frame launch
  const CameraBasis* cams;     // device array of n_frames frames, or null (use cam0)
  uint32_t n_frames;
  uint32_t width, height, max_depth, max_steps, flags;
  float light[3], light_intensity, eps_rel, ambient, background[3];
  float4* out;
  pr_aov* aov;
  unsigned long long* counter;
  unsigned long long* work;   // non-null: instrumented variant, adds WorkCounters
  bool analytic_small;        // analytic shaders only and stack need <= kShortStackDepth
  bool ahs_march;             // an any-hit shader on a sphere-traced shader: kernels with the any-hit march
};
int launch_trace(const TraceLaunch& L, cudaStream_t s);
// Camera frame of a pinhole camera for a width x height image (host, double
// precision rounded to float): every path computes its frames here, so one
// camera gives the same rays in pr_trace, pr_trace_frames and batches.
CameraBasis camera_frame(const pr_camera& cam, uint32_t width, uint32_t height);

}  // namespace pr

// Accessors the batch path needs from a scene (api.cu).
pr::SceneView pr_internal_view(const pr_scene* s);
bool pr_internal_built(const pr_scene* s);
// The scene has an any-hit shader on a sphere-traced intersection shader (its
// pixels need the kernels compiled with the any-hit march).
bool pr_internal_ahs_march(const pr_scene* s);
// Validate a description and give the device bytes pr_scene_create would
// allocate for it (pr_scene_device_bytes of the new scene) and the bytes of its
// inputs (the staging copy), without allocating.
pr_status pr_internal_scene_bytes(const pr_scene_desc* desc, size_t* bytes, size_t* input_bytes);
// pr_scene_create whose inputs go up through the caller's pinned buffer
// `staging` (at least the input bytes; the caller reuses it only after the
// copy on `stream` is done) instead of a pinned buffer of the scene's own,
// for a description already validated by pr_internal_scene_bytes (its
// per-element value checks are not repeated).
pr_status pr_internal_scene_create_staged(const pr_scene_desc* desc, cudaStream_t stream, void* staging,
                                          size_t staging_bytes, pr_scene** out);
// Completion flags for the next pr_trace_batch[_graph] of this batch: when
// the last tile of request r is written, the kernel stores seq into notify[r]
// (host-mapped memory, at least n requests). Only the megakernel modes write
// them; returns false (and sets nothing) for the four-stage wavefront.
struct pr_batch;
bool pr_internal_batch_notify(pr_batch* b, uint32_t* notify, uint32_t seq);
void pr_internal_set_error(const std::string& msg);

namespace pr {

}  // namespace pr
