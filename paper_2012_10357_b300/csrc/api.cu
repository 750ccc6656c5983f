// C ABI of the procedural ray tracer (declared in include/proceduray.h).
//
// Host responsibilities: validate descriptions, flatten the paper's entity
// model (BLAS -> geometries -> AABB primitives; Section 3.1.5) into leaf
// arrays, size one device arena per scene, copy inputs, and enqueue kernels.
// All per-ray and per-node work runs in the kernels of bvh.cu and trace.cu.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/proceduray.h"
#include "internal.h"

using namespace pr;

namespace {

thread_local std::string g_last_error;

pr_status fail(pr_status st, const std::string& msg) {
  g_last_error = msg;
  return st;
}

pr_status cuda_fail(cudaError_t e, const char* what) {
  g_last_error = std::string(what) + ": " + cudaGetErrorString(e);
  return e == cudaErrorMemoryAllocation ? PR_ERR_OUT_OF_MEMORY : PR_ERR_CUDA;
}

#define PR_CUDA(call, what)                   \
  do {                                        \
    cudaError_t e_ = (call);                  \
    if (e_ != cudaSuccess) return cuda_fail(e_, what); \
  } while (0)

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

constexpr uint32_t kTlas4MinInstances = 64;
// Scenes with at most this many BLAS levels (all small) and a small TLAS are
// built by one single-CTA launch.
constexpr uint32_t kFusedBuildMaxBlas = 32;

// Counts and host-side flattening of a description.
struct Layout {
  uint32_t n_prims, n_geoms, n_blas, n_inst, n_hg, n_mat, n_rec, n_rt, m;
  uint32_t n_vert = 0, n_tri = 0;
  std::vector<uint8_t> blas_tri;     // 1 if the BLAS holds triangles
  std::vector<uint32_t> leaf_prim;   // flattened BLAS leaves
  std::vector<uint32_t> leaf_gq;     // pairs (g, q)
  std::vector<int> blas_info;        // 4 ints per BLAS
  uint32_t n_leaves = 0, n_blas_nodes = 0, max_large = 0;
  // every hit group's intersection shader is analytic (sphere, box, pac-man) or
  // absent (triangles): no sphere tracing anywhere in the scene
  bool analytic_only = true;
  bool ahs_march = false;   // an any-hit shader on a sphere-traced intersection shader
  // bound on the traversal stack entries of any ray: a binary tree of n
  // leaves is at most n - 1 deep and a ray holds at most one entry per level
  // of the TLAS and of one BLAS below it
  uint32_t stack_bound = 0;
};

// check = false skips the per-element value checks (finite AABBs and
// vertices, index ranges, invertible transforms, record ranges) of a
// description already validated (the serving loop's copy, checked at submit);
// counts and ranges needed to flatten it are always checked.
pr_status validate_and_flatten(const pr_scene_desc* d, Layout& L, bool check = true) {
  if (!d) return fail(PR_ERR_INVALID_ARG, "null scene description");
  if (d->struct_size != sizeof(pr_scene_desc))
    return fail(PR_ERR_INVALID_ARG, "pr_scene_desc.struct_size mismatch (ABI version)");
  L.n_prims = d->n_prims;
  L.n_geoms = d->n_geoms;
  L.n_blas = d->n_blas;
  L.n_inst = d->n_inst;
  L.n_hg = d->n_hit_groups;
  L.n_mat = d->n_materials;
  L.n_rec = d->n_records;
  L.n_rt = d->n_ray_types;
  L.m = d->sbt_stride_m;
  if (L.n_rt < 2) return fail(PR_ERR_INVALID_ARG, "need ray types 0 (radiance) and 1 (shadow)");
  if (L.n_inst && (!L.n_blas || !L.n_geoms || !L.n_prims))
    return fail(PR_ERR_INVALID_ARG, "instances without BLAS/geometry/primitives");
  if (L.n_prims > (1u << 28) || L.n_inst > (1u << 28)) return fail(PR_ERR_INVALID_ARG, "too many primitives/instances (max 2^28)");
  auto need = [&](const void* p, uint32_t n, const char* name) -> bool {
    if (n && !p) {
      g_last_error = std::string("null array: ") + name;
      return false;
    }
    return true;
  };
  if (!need(d->aabbs, L.n_prims, "aabbs") || !need(d->params, L.n_prims, "params") ||
      !need(d->geom_prim_begin, L.n_geoms, "geom_prim_begin") || !need(d->geom_prim_count, L.n_geoms, "geom_prim_count") ||
      !need(d->blas_geom_begin, L.n_blas, "blas_geom_begin") || !need(d->blas_geom_count, L.n_blas, "blas_geom_count") ||
      !need(d->inst_xform, L.n_inst, "inst_xform") || !need(d->inst_blas, L.n_inst, "inst_blas") ||
      !need(d->inst_id, L.n_inst, "inst_id") || !need(d->inst_sbt_offset, L.n_inst, "inst_sbt_offset") ||
      !need(d->inst_mask, L.n_inst, "inst_mask") || !need(d->hit_groups, L.n_hg, "hit_groups") ||
      !need(d->materials, L.n_mat, "materials") || !need(d->sbt, L.n_rec, "sbt") ||
      !need(d->ray_types, L.n_rt, "ray_types"))
    return PR_ERR_INVALID_ARG;
  for (uint32_t p = 0; check && p < L.n_prims; ++p) {
    const float* b = d->aabbs + 6 * (size_t)p;
    for (int k = 0; k < 3; ++k)
      if (!(std::isfinite(b[k]) && std::isfinite(b[3 + k]) && b[k] <= b[3 + k]))
        return fail(PR_ERR_INVALID_ARG, "AABB " + std::to_string(p) + " not finite or lo > hi");
  }
  L.n_vert = d->n_vertices;
  L.n_tri = d->n_triangles;
  if ((L.n_vert && !d->vertices) || (L.n_tri && !d->indices))
    return fail(PR_ERR_INVALID_ARG, "null vertices/indices");
  if (L.n_vert > (1u << 28) || L.n_tri > (1u << 28)) return fail(PR_ERR_INVALID_ARG, "too many vertices/triangles");
  for (uint32_t v = 0; check && v < 3 * L.n_vert; ++v)
    if (!std::isfinite(d->vertices[v])) return fail(PR_ERR_INVALID_ARG, "vertex not finite");
  for (uint32_t t = 0; check && t < 3 * L.n_tri; ++t)
    if (d->indices[t] >= L.n_vert) return fail(PR_ERR_INVALID_ARG, "triangle vertex index out of range");
  auto is_tri = [&](uint32_t g) { return d->geom_type && d->geom_type[g] == PR_GEOM_TRIANGLES; };
  for (uint32_t g = 0; g < L.n_geoms; ++g) {
    if (d->geom_type && d->geom_type[g] != PR_GEOM_AABBS && d->geom_type[g] != PR_GEOM_TRIANGLES)
      return fail(PR_ERR_INVALID_ARG, "unknown geometry type");
    uint64_t e = (uint64_t)d->geom_prim_begin[g] + d->geom_prim_count[g];
    if (d->geom_prim_count[g] == 0 || e > (is_tri(g) ? L.n_tri : L.n_prims))
      return fail(PR_ERR_INVALID_ARG, "geometry " + std::to_string(g) + " primitive range empty or out of bounds");
  }
  L.blas_info.assign(4 * (size_t)L.n_blas, 0);
  L.blas_tri.assign(L.n_blas, 0);
  uint32_t max_geoms = 0;
  for (uint32_t b = 0; b < L.n_blas; ++b) {
    uint64_t e = (uint64_t)d->blas_geom_begin[b] + d->blas_geom_count[b];
    if (d->blas_geom_count[b] == 0 || e > L.n_geoms)
      return fail(PR_ERR_INVALID_ARG, "BLAS " + std::to_string(b) + " geometry range empty or out of bounds");
    max_geoms = std::max(max_geoms, d->blas_geom_count[b]);
    const bool tri = is_tri(d->blas_geom_begin[b]);
    for (uint32_t g = 1; g < d->blas_geom_count[b]; ++g)
      if (is_tri(d->blas_geom_begin[b] + g) != tri)
        return fail(PR_ERR_INVALID_ARG, "BLAS " + std::to_string(b) + " mixes triangle and AABB geometries");
    L.blas_tri[b] = tri ? 1 : 0;
    uint32_t first = L.n_leaves;
    for (uint32_t g = 0; g < d->blas_geom_count[b]; ++g) {
      uint32_t geom = d->blas_geom_begin[b] + g;
      for (uint32_t q = 0; q < d->geom_prim_count[geom]; ++q) {
        L.leaf_prim.push_back(d->geom_prim_begin[geom] + q);
        L.leaf_gq.push_back(g);
        L.leaf_gq.push_back(q);
        ++L.n_leaves;
      }
    }
    uint32_t n = L.n_leaves - first;
    // leaf refs keep bits 29..31 for their kind (kLoopBit, kTriBit, kLeafBit)
    if (L.n_leaves >= (1u << 29)) return fail(PR_ERR_INVALID_ARG, "too many BLAS leaves (max 2^29 - 1)");
    L.blas_info[4 * b + 0] = (int)L.n_blas_nodes;
    L.blas_info[4 * b + 1] = (int)first;
    L.blas_info[4 * b + 2] = (int)n;
    L.blas_info[4 * b + 3] = n == 1 ? (int)(kLeafBit | (tri ? kTriBit : 0u) | first)
                             : (!tri && n <= kLoopMaxLeaves && first + n <= (1u << 27))
                                 ? (int)(kLeafBit | kLoopBit | ((n - 1) << 27) | first)
                                 : 0;
    L.n_blas_nodes += n - 1;
    if (n > kSmallMax) L.max_large = std::max(L.max_large, n);
    L.stack_bound = std::max(L.stack_bound, n - 1);
  }
  L.stack_bound += L.n_inst ? L.n_inst - 1 : 0;
  if (L.n_inst > kSmallMax) L.max_large = std::max(L.max_large, L.n_inst);
  uint64_t max_index = 0;
  for (uint32_t k = 0; check && k < L.n_inst; ++k) {
    if (d->inst_blas[k] >= L.n_blas) return fail(PR_ERR_INVALID_ARG, "instance " + std::to_string(k) + " BLAS out of range");
    const float* x = d->inst_xform + 12 * (size_t)k;
    for (int i = 0; i < 12; ++i)
      if (!std::isfinite(x[i])) return fail(PR_ERR_INVALID_ARG, "instance transform not finite");
    double det = (double)x[0] * ((double)x[5] * x[10] - (double)x[6] * x[9]) -
                 (double)x[1] * ((double)x[4] * x[10] - (double)x[6] * x[8]) +
                 (double)x[2] * ((double)x[4] * x[9] - (double)x[5] * x[8]);
    if (!(std::fabs(det) > 1e-30)) return fail(PR_ERR_INVALID_ARG, "instance transform not invertible");
    uint64_t mi = (uint64_t)d->inst_sbt_offset[k] + (uint64_t)L.m * (d->blas_geom_count[d->inst_blas[k]] - 1) + L.n_rt;
    max_index = std::max(max_index, mi);
  }
  if (max_index >= (1ull << 31)) return fail(PR_ERR_INVALID_ARG, "Eq. 1 indices would exceed 2^31");
  for (uint32_t h = 0; h < L.n_hg; ++h) {
    uint32_t is = d->hit_groups[3 * h], chs = d->hit_groups[3 * h + 1], ahs = d->hit_groups[3 * h + 2];
    if (is != PR_NONE && is >= PR_IS_COUNT) return fail(PR_ERR_INVALID_ARG, "unknown intersection shader id");
    if (chs != PR_NONE && chs != PR_CHS_LAMBERT) return fail(PR_ERR_INVALID_ARG, "unknown closest-hit shader id");
    if (ahs != PR_NONE && ahs != PR_AHS_CUTOUT) return fail(PR_ERR_INVALID_ARG, "unknown any-hit shader id");
    if (ahs == PR_AHS_CUTOUT && is == PR_NONE)
      return fail(PR_ERR_INVALID_ARG, "any-hit shaders need an intersection shader");
    if (is != PR_NONE && is != PR_IS_SPHERE && is != PR_IS_BOX && is != PR_IS_PACMAN) L.analytic_only = false;
    if (ahs != PR_NONE && is >= PR_IS_TORUS && is <= PR_IS_JULIA_CUT) L.ahs_march = true;
  }
  for (uint32_t r = 0; check && r < L.n_rec; ++r) {
    if (d->sbt[4 * r] >= L.n_hg) return fail(PR_ERR_INVALID_ARG, "record " + std::to_string(r) + " hit group out of range");
    if (d->sbt[4 * r + 1] >= L.n_mat) return fail(PR_ERR_INVALID_ARG, "record " + std::to_string(r) + " material out of range");
  }
  for (uint32_t r = 0; r < L.n_rt; ++r)
    if (d->ray_types[2 * r] != PR_MISS_BACKGROUND && d->ray_types[2 * r] != PR_MISS_SHADOW)
      return fail(PR_ERR_INVALID_ARG, "unknown miss shader id");
  return PR_OK;
}

}  // namespace

struct pr_scene {
  Layout L;
  uint64_t serial = 0;   // unique per created scene (a freed address may be reused, a serial never is)
  char* arena = nullptr;
  size_t arena_bytes = 0;
  // pinned mirror of the arena's input prefix: an upload packs the inputs here
  // and sends them with one asynchronous copy
  char* h_stage = nullptr;
  size_t stage_bytes = 0;
  cudaEvent_t stage_done = nullptr;   // the last upload's copy has read h_stage
  // inputs
  float* aabbs;
  float4* params;
  float* xform;
  uint32_t *inst_blas, *inst_id, *inst_sbt, *inst_mask;
  float4* materials;
  uint4* sbt;                        // resolved shader records: is, chs, ahs, material
  uint2* ray_types;
  uint32_t* leaf_prim;
  uint2* leaf_gq;
  int4* blas_info;
  float* vertices;
  uint32_t* indices;
  float* tri_boxes;
  // BVH
  float4* blas_box;
  float4* blas_nodes;
  uint32_t *blas_perm, *blas_codes;
  float4* inst_rec;                  // [n_inst][6] instance records (see SceneView)
  float* inst_boxes;
  float4* tlas_nodes;
  float4* tlas4;                     // 4-wide TLAS collapsed from tlas_nodes
  uint32_t *c4_parent, *c4_even, *c4_rank;
  uint32_t* wide_slots;              // [8 (n_inst - 1) + 1] greedy collapse slots, then the frontier count
  float4* tlas8f = nullptr;          // float 8-wide TLAS nodes (allocated by the first such build)
  int tlas_format = 0;               // wide TLAS of the last build: 0 (depth-parity 4-wide), kWide4 (greedy), kWide8, kWide8Q
  uint32_t *tlas_perm, *tlas_codes;
  float* scene_box;
  uint32_t* error_word;
  // build
  BuildScratch scratch;
  LevelDesc* d_jobs;
  std::vector<LevelDesc> small_jobs;    // BLAS jobs (+ TLAS if small), in order: BLAS first
  std::vector<LevelDesc> large_blas;    // big BLAS levels
  LevelDesc tlas_job;
  bool tlas_small = true;
  bool built = false;
  // frame cameras
  CameraBasis* d_frames = nullptr;     // camera frames of a multi-frame launch
  uint32_t cams_cap = 0;
  std::vector<CameraBasis> h_frames;   // host staging of the frames
  int build_launches = 0;
  int trace_launches = 0;
};

namespace {

struct Carver {
  size_t off = 0;
  template <typename T>
  size_t take(size_t count) {
    size_t o = off;
    off = align256(off + sizeof(T) * (count ? count : 1));
    return o;
  }
};

// Byte offsets of every buffer in a scene's device arena (256-byte aligned);
// the inputs form the prefix [0, o_tbox), copied to the device in one piece.
struct ArenaPlan {
  size_t o_aabbs, o_params, o_xform, o_iblas, o_iid, o_isbt, o_imask, o_mat, o_sbt, o_rt, o_lp, o_lgq, o_binfo,
      o_vert, o_idx;
  size_t o_tbox, o_bbox, o_bnodes, o_bperm, o_bcodes, o_rec, o_iboxes, o_tnodes, o_t4, o_c4p, o_c4e, o_c4r, o_wide, o_tperm,
      o_tcodes, o_sbox, o_err;
  size_t o_k0, o_k1, o_v0, o_v1, o_hist, o_cnt, o_pi, o_pl, o_part, o_jobs;
  size_t total;
};

ArenaPlan plan_arena(const Layout& L) {
  Carver c;
  ArenaPlan P;
  P.o_aabbs = c.take<float>(6 * (size_t)L.n_prims);
  P.o_params = c.take<float4>(4 * (size_t)L.n_prims);
  P.o_xform = c.take<float>(12 * (size_t)L.n_inst);
  P.o_iblas = c.take<uint32_t>(L.n_inst);
  P.o_iid = c.take<uint32_t>(L.n_inst);
  P.o_isbt = c.take<uint32_t>(L.n_inst);
  P.o_imask = c.take<uint32_t>(L.n_inst);
  P.o_mat = c.take<float4>(L.n_mat);
  P.o_sbt = c.take<uint4>(L.n_rec);
  P.o_rt = c.take<uint2>(L.n_rt);
  P.o_lp = c.take<uint32_t>(L.n_leaves);
  P.o_lgq = c.take<uint2>(L.n_leaves);
  P.o_binfo = c.take<int4>(L.n_blas);
  P.o_vert = c.take<float>(3 * (size_t)L.n_vert);
  P.o_idx = c.take<uint32_t>(3 * (size_t)L.n_tri);
  // everything above is input (one prefix of the arena, copied in one piece)
  const size_t ni = L.n_inst ? L.n_inst - 1 : 0;
  P.o_tbox = c.take<float>(6 * (size_t)L.n_tri);
  P.o_bbox = c.take<float4>(2 * (size_t)L.n_blas);
  P.o_bnodes = c.take<float4>(4 * (size_t)L.n_blas_nodes);
  P.o_bperm = c.take<uint32_t>(L.n_leaves);
  P.o_bcodes = c.take<uint32_t>(L.n_leaves);
  P.o_rec = c.take<float4>(6 * (size_t)L.n_inst);
  P.o_iboxes = c.take<float>(6 * (size_t)L.n_inst);
  P.o_tnodes = c.take<float4>(4 * ni);
  P.o_t4 = c.take<float4>(8 * ni);
  P.o_c4p = c.take<uint32_t>(L.n_inst);
  P.o_c4e = c.take<uint32_t>(L.n_inst);
  P.o_c4r = c.take<uint32_t>(L.n_inst);
  P.o_wide = c.take<uint32_t>(8 * ni + 1);
  P.o_tperm = c.take<uint32_t>(L.n_inst);
  P.o_tcodes = c.take<uint32_t>(L.n_inst);
  P.o_sbox = c.take<float>(8);
  P.o_err = c.take<uint32_t>(1);
  const uint32_t nl = L.max_large;
  P.o_k0 = c.take<uint32_t>(nl);
  P.o_k1 = c.take<uint32_t>(nl);
  P.o_v0 = c.take<uint32_t>(nl);
  P.o_v1 = c.take<uint32_t>(nl);
  P.o_hist = c.take<uint32_t>(256 * (size_t)sort_tiles(nl));
  P.o_cnt = c.take<uint32_t>(nl);
  P.o_pi = c.take<uint32_t>(nl);
  P.o_pl = c.take<uint32_t>(nl);
  P.o_part = c.take<float>(6 * (size_t)kMaxPartials);
  P.o_jobs = c.take<LevelDesc>((size_t)L.n_blas + 1);
  P.total = c.off;
  return P;
}

// Pack the inputs into a pinned staging buffer (the scene's own, allocated on
// first use, or `ext`, a caller's buffer of at least stage_bytes whose reuse
// the caller orders after this copy) and send them with one asynchronous copy.
pr_status upload(pr_scene* s, const pr_scene_desc* d, cudaStream_t st, char* ext = nullptr) {
  const Layout& L = s->L;
  // the previous upload's copy must have read the staging buffer before it is refilled
  PR_CUDA(cudaEventSynchronize(s->stage_done), "wait for the previous upload");
  if (!ext && !s->h_stage) PR_CUDA(cudaMallocHost(&s->h_stage, s->stage_bytes), "pinned staging buffer");
  char* H = ext ? ext : s->h_stage;
  auto put = [&](const void* dev_dst, const void* src, size_t bytes) {
    if (bytes) std::memcpy(H + (static_cast<const char*>(dev_dst) - s->arena), src, bytes);
  };
  put(s->aabbs, d->aabbs, sizeof(float) * 6 * L.n_prims);
  put(s->params, d->params, sizeof(float) * PR_PARAMS_PER_PRIM * L.n_prims);
  put(s->xform, d->inst_xform, sizeof(float) * 12 * L.n_inst);
  put(s->inst_blas, d->inst_blas, sizeof(uint32_t) * L.n_inst);
  put(s->inst_id, d->inst_id, sizeof(uint32_t) * L.n_inst);
  put(s->inst_sbt, d->inst_sbt_offset, sizeof(uint32_t) * L.n_inst);
  put(s->inst_mask, d->inst_mask, sizeof(uint32_t) * L.n_inst);
  put(s->materials, d->materials, sizeof(float) * 4 * L.n_mat);
  // Device shader records hold what a DXR shader record holds: the hit group's
  // shader identifiers (intersection, closest-hit, any-hit) and the record's
  // local argument (its material), so one 16-byte load per Eq. 1 lookup gives
  // the shaders to run (the hit-group indices were validated above).
  uint32_t* rec = reinterpret_cast<uint32_t*>(H + (reinterpret_cast<const char*>(s->sbt) - s->arena));
  for (uint32_t r = 0; r < L.n_rec; ++r) {
    const uint32_t h = d->sbt[4 * r];
    for (int k = 0; k < 3; ++k) rec[4 * r + k] = d->hit_groups[3 * h + k];
    rec[4 * r + 3] = d->sbt[4 * r + 1];
  }
  put(s->ray_types, d->ray_types, sizeof(uint32_t) * 2 * L.n_rt);
  put(s->leaf_prim, L.leaf_prim.data(), sizeof(uint32_t) * L.n_leaves);
  put(s->leaf_gq, L.leaf_gq.data(), sizeof(uint32_t) * 2 * L.n_leaves);
  put(s->blas_info, L.blas_info.data(), sizeof(int) * 4 * L.n_blas);
  put(s->vertices, d->vertices, sizeof(float) * 3 * L.n_vert);
  put(s->indices, d->indices, sizeof(uint32_t) * 3 * L.n_tri);
  PR_CUDA(cudaMemcpyAsync(s->arena, H, s->stage_bytes, cudaMemcpyHostToDevice, st), "copy scene inputs");
  PR_CUDA(cudaEventRecord(s->stage_done, st), "record upload");
  s->built = false;
  return PR_OK;
}

SceneView view_of(const pr_scene* s) {
  SceneView v;
  v.inst_rec = s->inst_rec;
  v.tlas_nodes = s->tlas_nodes;
  v.tlas_root_ref = s->L.n_inst == 1 ? (int)kLeafBit : 0;
  // the 4-wide TLAS pays off on large instance counts only (measured: +3 % at
  // 100 000 instances, -7 % at 5); small TLASes keep the binary traversal
  const bool wide = s->L.n_inst >= kTlas4MinInstances;
  v.tlas4 = wide && s->tlas_format != kWide8 && s->tlas_format != kWide8Q ? s->tlas4 : nullptr;
  v.tlas8 = !wide ? nullptr : s->tlas_format == kWide8Q ? s->tlas4 : s->tlas_format == kWide8 ? s->tlas8f : nullptr;
  v.tlas8_format = v.tlas8 ? s->tlas_format : 0;
  v.tlas4_root = v.tlas_root_ref;
  v.scene_box = s->scene_box;
  v.blas_info = s->blas_info;
  v.blas_box = s->blas_box;
  v.blas_nodes = s->blas_nodes;
  v.leaf_prim = s->leaf_prim;
  v.leaf_gq = s->leaf_gq;
  v.vertices = s->vertices;
  v.indices = s->indices;
  v.aabbs = s->aabbs;
  v.params = s->params;
  v.sbt = s->sbt;
  v.materials = s->materials;
  v.ray_types = s->ray_types;
  v.n_inst = s->L.n_inst;
  v.n_blas = s->L.n_blas;
  v.n_records = s->L.n_rec;
  v.sbt_stride_m = s->L.m;
  v.error_word = s->error_word;
  return v;
}

bool params_ok(const pr_trace_params* p) {
  if (!p || p->struct_size != sizeof(pr_trace_params)) {
    g_last_error = "pr_trace_params null or struct_size mismatch";
    return false;
  }
  if (p->width == 0 || p->height == 0 || p->width > 65536 || p->height > 65536 || p->max_depth < 1 ||
      p->max_depth > 2 || p->max_steps == 0) {
    g_last_error = "bad trace params (size 1..65536, max_depth 1..2, max_steps >= 1)";
    return false;
  }
  return true;
}

}  // namespace

namespace pr {

size_t build_scratch_bytes(uint32_t n) {
  Carver c;
  for (int k = 0; k < 4; ++k) c.take<uint32_t>(n);
  c.take<uint32_t>(256 * (size_t)sort_tiles(n));
  for (int k = 0; k < 3; ++k) c.take<uint32_t>(n);
  c.take<float>(6 * (size_t)kMaxPartials);
  return c.off;
}

BuildScratch carve_build_scratch(void* base, uint32_t n) {
  Carver c;
  char* A = (char*)base;
  BuildScratch sc;
  sc.keys[0] = (uint32_t*)(A + c.take<uint32_t>(n));
  sc.keys[1] = (uint32_t*)(A + c.take<uint32_t>(n));
  sc.vals[0] = (uint32_t*)(A + c.take<uint32_t>(n));
  sc.vals[1] = (uint32_t*)(A + c.take<uint32_t>(n));
  sc.hist = (uint32_t*)(A + c.take<uint32_t>(256 * (size_t)sort_tiles(n)));
  sc.counters = (uint32_t*)(A + c.take<uint32_t>(n));
  sc.parent_int = (uint32_t*)(A + c.take<uint32_t>(n));
  sc.parent_leaf = (uint32_t*)(A + c.take<uint32_t>(n));
  sc.partial = (float*)(A + c.take<float>(6 * (size_t)kMaxPartials));
  sc.cluster_boxes = nullptr;
  sc.max_n = n;
  return sc;
}

// Pinhole camera frame (Section 2.2.3's ray generation, vertical field of
// view): forward = unit(look_at - eye), right = unit(up x forward), the image's
// up = forward x right; pixel (x, y) of a W x H image maps to
// ndc = ((x + 0.5) * 2 / W - 1) * tan(fov / 2) * W / H and
// ((y + 0.5) * 2 / H - 1) * (-tan(fov / 2)) in camera_ray. Double precision,
// rounded once to float.
CameraBasis camera_frame(const pr_camera& c, uint32_t width, uint32_t height) {
  double e[3], f[3], u[3], r[3], v[3];
  for (int k = 0; k < 3; ++k) {
    e[k] = c.eye[k];
    f[k] = (double)c.look_at[k] - e[k];
    u[k] = c.up[k];
  }
  auto unit = [](double* a) {
    const double l = std::sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]);
    for (int k = 0; k < 3; ++k) a[k] /= l;
  };
  auto cross = [](const double* a, const double* b, double* o) {
    o[0] = a[1] * b[2] - a[2] * b[1];
    o[1] = a[2] * b[0] - a[0] * b[2];
    o[2] = a[0] * b[1] - a[1] * b[0];
  };
  unit(f);
  cross(u, f, r);
  unit(r);
  cross(f, r, v);
  const double th = std::tan((double)c.vfov_deg * (3.14159265358979323846 / 360.0));
  CameraBasis b;
  b.eye = make_float3((float)e[0], (float)e[1], (float)e[2]);
  b.fwd = make_float3((float)f[0], (float)f[1], (float)f[2]);
  b.right = make_float3((float)r[0], (float)r[1], (float)r[2]);
  b.up = make_float3((float)v[0], (float)v[1], (float)v[2]);
  b.kx = 2.f / (float)width;
  b.ky = 2.f / (float)height;
  b.ax = (float)(th * ((double)width / (double)height));
  b.ay = (float)(-th);
  return b;
}

}  // namespace pr

pr::SceneView pr_internal_view(const pr_scene* s) { return view_of(s); }

pr_status pr_internal_scene_bytes(const pr_scene_desc* desc, size_t* bytes, size_t* input_bytes) {
  Layout L;
  pr_status st = validate_and_flatten(desc, L);
  if (st == PR_OK) {
    const ArenaPlan P = plan_arena(L);
    *bytes = P.total;
    if (input_bytes) *input_bytes = P.o_tbox;
  }
  return st;
}
bool pr_internal_built(const pr_scene* s) { return s && s->built; }
bool pr_internal_ahs_march(const pr_scene* s) { return s && s->L.ahs_march; }
void pr_internal_set_error(const std::string& msg) { g_last_error = msg; }

extern "C" {

uint32_t pr_version(void) { return PR_ABI_VERSION; }

const char* pr_last_error(void) { return g_last_error.c_str(); }

pr_status pr_scene_validate(const pr_scene_desc* desc) {
  Layout L;
  return validate_and_flatten(desc, L);
}

pr_status pr_sbt_index(uint32_t r, uint32_t m, uint32_t g, uint32_t i, uint32_t n_records, uint32_t* out) {
  uint64_t a = (uint64_t)r + (uint64_t)m * g + i;
  if (a >= n_records) return fail(PR_ERR_SBT_INDEX, "Eq. 1 index outside the shader table");
  if (out) *out = (uint32_t)a;
  return PR_OK;
}

}  // extern "C"

namespace {

// pr_scene_create; with `ext` (pinned, at least the scene's input bytes) the
// inputs go up through that buffer and the scene gets no staging buffer of its
// own until a later pr_scene_upload.
pr_status create_scene(const pr_scene_desc* desc, cudaStream_t stream, char* ext, size_t ext_bytes, pr_scene** out,
                       bool check = true) {
  if (!out) return fail(PR_ERR_INVALID_ARG, "null output pointer");
  *out = nullptr;
  pr_scene* s = new pr_scene();
  static std::atomic<uint64_t> next_serial{1};
  s->serial = next_serial.fetch_add(1);
  pr_status vs = validate_and_flatten(desc, s->L, check);
  if (vs != PR_OK) {
    delete s;
    return vs;
  }
  const Layout& L = s->L;
  const ArenaPlan P = plan_arena(L);
  s->arena_bytes = P.total;
  s->stage_bytes = P.o_tbox;
  if (ext && ext_bytes < s->stage_bytes) {
    delete s;
    return fail(PR_ERR_INVALID_ARG, "staging buffer smaller than the scene's inputs");
  }
  cudaError_t e = cudaMalloc(&s->arena, s->arena_bytes);
  if (e == cudaSuccess && !ext) e = cudaMallocHost(&s->h_stage, s->stage_bytes);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->stage_done, cudaEventDisableTiming);
  if (e != cudaSuccess) {
    pr_scene_destroy(s);
    return cuda_fail(e, "scene arena / pinned staging buffer");
  }
  char* A = s->arena;
  s->aabbs = (float*)(A + P.o_aabbs);
  s->params = (float4*)(A + P.o_params);
  s->xform = (float*)(A + P.o_xform);
  s->inst_blas = (uint32_t*)(A + P.o_iblas);
  s->inst_id = (uint32_t*)(A + P.o_iid);
  s->inst_sbt = (uint32_t*)(A + P.o_isbt);
  s->inst_mask = (uint32_t*)(A + P.o_imask);
  s->materials = (float4*)(A + P.o_mat);
  s->sbt = (uint4*)(A + P.o_sbt);
  s->ray_types = (uint2*)(A + P.o_rt);
  s->leaf_prim = (uint32_t*)(A + P.o_lp);
  s->leaf_gq = (uint2*)(A + P.o_lgq);
  s->blas_info = (int4*)(A + P.o_binfo);
  s->vertices = (float*)(A + P.o_vert);
  s->indices = (uint32_t*)(A + P.o_idx);
  s->tri_boxes = (float*)(A + P.o_tbox);
  s->blas_box = (float4*)(A + P.o_bbox);
  s->blas_nodes = (float4*)(A + P.o_bnodes);
  s->blas_perm = (uint32_t*)(A + P.o_bperm);
  s->blas_codes = (uint32_t*)(A + P.o_bcodes);
  s->inst_rec = (float4*)(A + P.o_rec);
  s->inst_boxes = (float*)(A + P.o_iboxes);
  s->tlas_nodes = (float4*)(A + P.o_tnodes);
  s->tlas4 = (float4*)(A + P.o_t4);
  s->c4_parent = (uint32_t*)(A + P.o_c4p);
  s->c4_even = (uint32_t*)(A + P.o_c4e);
  s->c4_rank = (uint32_t*)(A + P.o_c4r);
  s->wide_slots = (uint32_t*)(A + P.o_wide);
  s->tlas_perm = (uint32_t*)(A + P.o_tperm);
  s->tlas_codes = (uint32_t*)(A + P.o_tcodes);
  s->scene_box = (float*)(A + P.o_sbox);
  s->error_word = (uint32_t*)(A + P.o_err);
  s->scratch.keys[0] = (uint32_t*)(A + P.o_k0);
  s->scratch.keys[1] = (uint32_t*)(A + P.o_k1);
  s->scratch.vals[0] = (uint32_t*)(A + P.o_v0);
  s->scratch.vals[1] = (uint32_t*)(A + P.o_v1);
  s->scratch.hist = (uint32_t*)(A + P.o_hist);
  s->scratch.counters = (uint32_t*)(A + P.o_cnt);
  s->scratch.parent_int = (uint32_t*)(A + P.o_pi);
  s->scratch.parent_leaf = (uint32_t*)(A + P.o_pl);
  s->scratch.partial = (float*)(A + P.o_part);
  s->scratch.cluster_boxes = nullptr;
  s->scratch.max_n = s->L.max_large;
  s->d_jobs = (LevelDesc*)(A + P.o_jobs);

  // Level jobs: BLAS levels (small ones in one launch, large ones separately), then the TLAS.
  for (uint32_t b = 0; b < L.n_blas; ++b) {
    LevelDesc J;
    J.boxes = L.blas_tri[b] ? s->tri_boxes : s->aabbs;
    J.gather = s->leaf_prim + L.blas_info[4 * b + 1];
    J.n = (uint32_t)L.blas_info[4 * b + 2];
    J.leaf_ref_base = (uint32_t)L.blas_info[4 * b + 1] | (L.blas_tri[b] ? kTriBit : 0u);
    J.nodes = s->blas_nodes + 4 * (size_t)L.blas_info[4 * b + 0];
    J.perm = s->blas_perm + L.blas_info[4 * b + 1];
    J.codes = s->blas_codes + L.blas_info[4 * b + 1];
    J.root_box = (float*)(s->blas_box + 2 * (size_t)b);
    if (J.n > kSmallMax) s->large_blas.push_back(J);
    else s->small_jobs.push_back(J);
  }
  LevelDesc T;
  T.boxes = s->inst_boxes;
  T.gather = nullptr;
  T.n = L.n_inst;
  T.leaf_ref_base = 0;
  T.nodes = s->tlas_nodes;
  T.perm = s->tlas_perm;
  T.codes = s->tlas_codes;
  T.root_box = s->scene_box;
  s->tlas_job = T;
  s->tlas_small = L.n_inst <= kSmallMax;
  std::vector<LevelDesc> jobs = s->small_jobs;
  jobs.push_back(T);   // the TLAS job sits after the BLAS jobs (used when it is small)
  cudaStream_t st = stream;
  e = cudaMemcpyAsync(s->d_jobs, jobs.data(), sizeof(LevelDesc) * jobs.size(), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(s->error_word, 0, sizeof(uint32_t), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(s->scene_box, 0, 8 * sizeof(float), st);
  if (e != cudaSuccess) {
    pr_scene_destroy(s);
    return cuda_fail(e, "scene setup copy");
  }
  pr_status us = upload(s, desc, st, ext);
  if (us != PR_OK) {
    pr_scene_destroy(s);
    return us;
  }
  *out = s;
  return PR_OK;
}

}  // namespace

pr_status pr_internal_scene_create_staged(const pr_scene_desc* desc, cudaStream_t stream, void* staging,
                                          size_t staging_bytes, pr_scene** out) {
  return create_scene(desc, stream, static_cast<char*>(staging), staging_bytes, out, false);
}

extern "C" {

pr_status pr_scene_create(const pr_scene_desc* desc, void* stream, pr_scene** out) {
  return create_scene(desc, (cudaStream_t)stream, nullptr, 0, out);
}

pr_status pr_scene_upload(pr_scene* s, const pr_scene_desc* desc, void* stream) {
  if (!s) return fail(PR_ERR_INVALID_ARG, "null scene");
  Layout L;
  pr_status st = validate_and_flatten(desc, L);
  if (st != PR_OK) return st;
  if (L.n_prims != s->L.n_prims || L.n_geoms != s->L.n_geoms || L.n_blas != s->L.n_blas || L.n_inst != s->L.n_inst ||
      L.n_hg != s->L.n_hg || L.n_mat != s->L.n_mat || L.n_rec != s->L.n_rec || L.n_rt != s->L.n_rt ||
      L.blas_info != s->L.blas_info || L.n_vert != s->L.n_vert || L.n_tri != s->L.n_tri)
    return fail(PR_ERR_INVALID_ARG, "pr_scene_upload needs the same counts and BLAS layout as at creation");
  s->L = std::move(L);
  return upload(s, desc, (cudaStream_t)stream);
}

}  // extern "C"

namespace {

// Streams the builds of pr_build_bvh_many fan out to, one pool per device,
// created on first use and kept for the life of the process (64 field scenes:
// 0.97 / 0.91 / 0.89 ms with 8 / 16 / 32 streams).
constexpr int kBuildStreams = 32;
// A fan-out is a few hundred small launches; the pool keeps the last one as a
// CUDA graph and replays it while the same scenes are built with the same
// flags. A scene's launches (shapes and arguments) are fixed by its layout,
// which never changes after creation, so the graph re-runs every kernel of
// the builds on the scenes' current inputs.
#ifndef PR_BUILD_GRAPHS
#define PR_BUILD_GRAPHS 1
#endif
struct BuiltState {   // host-side state a build leaves in its scene
  int tlas_format, build_launches;
};
struct BuildPool {
  cudaStream_t streams[kBuildStreams] = {};
  cudaEvent_t done[kBuildStreams] = {};
  cudaEvent_t start = nullptr;
  cudaEvent_t ploc = nullptr;   // the previous PLOC clustering launch of the fan-out
  cudaStream_t capture = nullptr;
  cudaGraphExec_t graph = nullptr;
  std::vector<std::pair<const pr_scene*, uint64_t>> key;   // scenes (address, serial) of the graph, in order
  uint32_t key_flags = 0;
  std::vector<BuiltState> state;
  bool ready = false;
};

// Order of the cooperative clustering launches of one fan-out: each waits for
// the one before it (two cooperative grids are never resident side by side).
struct PlocChain {
  cudaEvent_t ev = nullptr;
  bool armed = false;
};

pr_status build_impl(pr_scene* s, uint32_t flags, cudaStream_t st, PlocChain* chain);

// Known flags, at most one wide-TLAS format.
bool build_flags_ok(uint32_t f) {
  const uint32_t wide = f & (PR_BUILD_TLAS_PARITY4 | PR_BUILD_TLAS_BVH8 | PR_BUILD_TLAS_BVH8_F32);
  return !(f & ~(PR_BUILD_TLAS_PLOC | PR_BUILD_TLAS_PARITY4 | PR_BUILD_TLAS_BVH8 | PR_BUILD_TLAS_BVH8_F32)) &&
         (wide & (wide - 1)) == 0;
}
std::mutex g_pool_mutex;
BuildPool g_pools[64];

}  // namespace

extern "C" {

pr_status pr_build_bvh_many(pr_scene* const* scenes, uint32_t n, void* stream) {
  return pr_build_bvh_many_ex(scenes, n, 0u, stream);
}

pr_status pr_build_bvh_many_ex(pr_scene* const* scenes, uint32_t n, uint32_t flags, void* stream) {
  if (!build_flags_ok(flags)) return fail(PR_ERR_INVALID_ARG, "unknown or conflicting build flags");
  if (n == 0) return PR_OK;
  if (!scenes) return fail(PR_ERR_INVALID_ARG, "null scene array");
  for (uint32_t i = 0; i < n; ++i)
    if (!scenes[i]) return fail(PR_ERR_INVALID_ARG, "null scene in the array");
  {
    // a scene listed twice would be built by two streams into one arena at once
    std::vector<pr_scene*> sorted(scenes, scenes + n);
    std::sort(sorted.begin(), sorted.end());
    if (std::adjacent_find(sorted.begin(), sorted.end()) != sorted.end())
      return fail(PR_ERR_INVALID_ARG, "a scene appears twice in the array");
  }
  cudaStream_t st = (cudaStream_t)stream;
  if (n == 1) return build_impl(scenes[0], flags, st, nullptr);
  int dev = 0;
  PR_CUDA(cudaGetDevice(&dev), "cudaGetDevice");
  if (dev < 0 || dev >= 64) return fail(PR_ERR_INVALID_ARG, "device ordinal beyond 63");
  std::lock_guard<std::mutex> lock(g_pool_mutex);   // one fan-out at a time per process
  BuildPool& P = g_pools[dev];
  if (!P.ready) {
    for (int k = 0; k < kBuildStreams; ++k) {
      PR_CUDA(cudaStreamCreateWithFlags(&P.streams[k], cudaStreamNonBlocking), "build stream");
      PR_CUDA(cudaEventCreateWithFlags(&P.done[k], cudaEventDisableTiming), "build event");
    }
    PR_CUDA(cudaEventCreateWithFlags(&P.start, cudaEventDisableTiming), "build event");
    PR_CUDA(cudaEventCreateWithFlags(&P.ploc, cudaEventDisableTiming), "build event");
    P.ready = true;
  }
  const int used = (int)std::min<uint32_t>(n, kBuildStreams);
  // the fan-out from stream `from` over the pool streams and back into it
  auto fan_out = [&](cudaStream_t from) -> pr_status {
    // fork: every pool stream waits for the work already on `from`
    PR_CUDA(cudaEventRecord(P.start, from), "record fork");
    for (int k = 0; k < used; ++k) PR_CUDA(cudaStreamWaitEvent(P.streams[k], P.start, 0), "fork");
    pr_status result = PR_OK;
    PlocChain chain{P.ploc, false};
    for (uint32_t i = 0; i < n; ++i) {
      const pr_status b = build_impl(scenes[i], flags, P.streams[i % kBuildStreams], &chain);
      if (b != PR_OK && result == PR_OK) result = b;
    }
    // join: `from` waits for every build
    for (int k = 0; k < used; ++k) {
      PR_CUDA(cudaEventRecord(P.done[k], P.streams[k]), "record join");
      PR_CUDA(cudaStreamWaitEvent(from, P.done[k], 0), "join");
    }
    return result;
  };
  // Graph replay: not for PLOC (cooperative launches chained by an event) nor
  // the float 8-wide format (its first build allocates), nor when the
  // caller's stream is itself being captured (the builds then join that capture).
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  PR_CUDA(cudaStreamIsCapturing(st, &cap), "cudaStreamIsCapturing");
  if (!PR_BUILD_GRAPHS || (flags & (PR_BUILD_TLAS_PLOC | PR_BUILD_TLAS_BVH8_F32)) || cap != cudaStreamCaptureStatusNone)
    return fan_out(st);
  std::vector<std::pair<const pr_scene*, uint64_t>> key(n);
  for (uint32_t i = 0; i < n; ++i) key[i] = {scenes[i], scenes[i]->serial};
  if (!P.graph || P.key_flags != flags || P.key != key) {
    if (P.graph) {
      cudaGraphExecDestroy(P.graph);
      P.graph = nullptr;
      P.key.clear();
    }
    // A capture that fails anywhere launched nothing (although the builds it
    // recorded marked their scenes built): the builds then run directly.
    if (!P.capture && cudaStreamCreateWithFlags(&P.capture, cudaStreamNonBlocking) != cudaSuccess) {
      P.capture = nullptr;
      cudaGetLastError();
      return fan_out(st);
    }
    if (cudaStreamBeginCapture(P.capture, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
      cudaGetLastError();
      return fan_out(st);
    }
    const pr_status r = fan_out(P.capture);
    cudaGraph_t g = nullptr;
    const cudaError_t ec = cudaStreamEndCapture(P.capture, &g);
    cudaError_t ei = cudaErrorUnknown;
    if (r == PR_OK && ec == cudaSuccess && g) ei = cudaGraphInstantiate(&P.graph, g, 0);
    if (g) cudaGraphDestroy(g);
    if (ei != cudaSuccess) {
      P.graph = nullptr;
      cudaGetLastError();
      return fan_out(st);
    }
    P.key = std::move(key);
    P.key_flags = flags;
    P.state.resize(n);
    for (uint32_t i = 0; i < n; ++i) P.state[i] = {scenes[i]->tlas_format, scenes[i]->build_launches};
  }
  const cudaError_t el = cudaGraphLaunch(P.graph, st);
  if (el != cudaSuccess) {
    for (uint32_t i = 0; i < n; ++i) scenes[i]->built = false;
    return cuda_fail(el, "build graph launch");
  }
  for (uint32_t i = 0; i < n; ++i) {
    scenes[i]->built = true;
    scenes[i]->tlas_format = P.state[i].tlas_format;
    scenes[i]->build_launches = P.state[i].build_launches;
  }
  return PR_OK;
}

pr_status pr_build_bvh(pr_scene* s, void* stream) { return pr_build_bvh_ex(s, 0u, stream); }

pr_status pr_build_bvh_ex(pr_scene* s, uint32_t flags, void* stream) {
  if (!build_flags_ok(flags)) return fail(PR_ERR_INVALID_ARG, "unknown or conflicting build flags");
  return build_impl(s, flags, (cudaStream_t)stream, nullptr);
}

}  // extern "C"

namespace {

pr_status build_impl(pr_scene* s, uint32_t flags, cudaStream_t st, PlocChain* chain) {
  if (!s) return fail(PR_ERR_INVALID_ARG, "null scene");
  int launches = 0;
  const InstanceArgs IA{s->xform, s->inst_blas, s->inst_id, s->inst_sbt, s->inst_mask, s->blas_box,
                        s->blas_info, s->L.n_inst, s->inst_boxes, s->inst_rec};
  if (s->L.n_tri == 0 && s->large_blas.empty() && s->L.n_inst > 0 && s->tlas_small &&
      s->small_jobs.size() <= kFusedBuildMaxBlas && s->L.n_inst < kTlas4MinInstances) {
    // small scene: BLAS levels, instances and TLAS in one single-CTA launch
    launches += launch_build_scene_small(s->d_jobs, (uint32_t)s->small_jobs.size(), IA, st);
  } else {
    // 0. triangle boxes (leaf input of triangle BLASes)
    launches += launch_triangle_boxes(s->vertices, s->indices, s->L.n_tri, s->tri_boxes, st);
    // 1. every small BLAS in one launch, one CTA each
    launches += launch_build_small(s->d_jobs, (uint32_t)s->small_jobs.size(), st);
    for (const LevelDesc& J : s->large_blas) launches += launch_build_large(J, s->scratch, st);
    // 2. instance world boxes, world->object transforms
    launches += launch_instances(IA, st);
    // 3. TLAS, then its 4-wide collapse
    if (s->L.n_inst > 0) {
      if (s->tlas_small) {
        launches += launch_build_small(s->d_jobs + s->small_jobs.size(), 1, st);
      } else if (flags & PR_BUILD_TLAS_PLOC) {
        BuildScratch sc = s->scratch;
        sc.cluster_boxes = reinterpret_cast<float*>(s->tlas4);   // 128 B per instance, free until the collapse
        const int k = launch_build_ploc(s->tlas_job, sc, s->error_word, st, chain && chain->armed ? chain->ev : nullptr,
                                        chain ? chain->ev : nullptr);
        if (k < 0) return cuda_fail(cudaGetLastError(), "PLOC TLAS build launch");
        if (chain) chain->armed = true;
        launches += k;
      } else {
        launches += launch_build_large(s->tlas_job, s->scratch, st);
      }
      // the wide TLAS is traversed from kTlas4MinInstances up; below that it is not built
      if (s->L.n_inst >= kTlas4MinInstances) {
        const int fmt = (flags & PR_BUILD_TLAS_BVH8) ? kWide8Q : (flags & PR_BUILD_TLAS_BVH8_F32) ? kWide8
                        : (flags & PR_BUILD_TLAS_PARITY4) ? 0 : kWide4;
        if (fmt == 0) {
          launches += launch_collapse4(s->tlas_nodes, s->L.n_inst, s->c4_parent, s->c4_even, s->c4_rank, s->tlas4, st);
        } else {
          float4* out = s->tlas4;   // 128 B per binary node: room for the 4-wide or quantised 8-wide nodes
          if (fmt == kWide8) {
            if (!s->tlas8f)
              PR_CUDA(cudaMalloc(&s->tlas8f, sizeof(float4) * 14 * (size_t)(s->L.n_inst - 1)), "8-wide TLAS nodes");
            out = s->tlas8f;
          }
          const WideScratch ws{s->wide_slots, s->c4_even, s->c4_rank, s->c4_parent,
                               s->wide_slots + 8 * (size_t)(s->L.n_inst - 1)};
          launches += launch_collapse_wide(s->tlas_nodes, s->L.n_inst, fmt, ws, out, s->error_word, st);
        }
        s->tlas_format = fmt;
      }
    }
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "BVH build launch");
  s->built = true;
  s->build_launches = launches;
  return PR_OK;
}

}  // namespace

extern "C" {

static pr_status trace_impl(pr_scene* s, const pr_camera* cam0, const CameraBasis* d_frames, uint32_t n_frames,
                            const pr_trace_params* p, float* out_rgba, pr_aov* out_aov, uint64_t* counter,
                            cudaStream_t st, uint64_t* work = nullptr) {
  TraceLaunch T;
  T.S = view_of(s);
  if (p->flags & PR_TRACE_TLAS_BVH2) {   // binary TLAS traversal (comparison)
    T.S.tlas4 = nullptr;
    T.S.tlas8 = nullptr;
  }
  T.cam0 = camera_frame(*cam0, p->width, p->height);
  T.cams = d_frames;
  T.n_frames = n_frames;
  T.width = p->width;
  T.height = p->height;
  T.max_depth = p->max_depth;
  T.max_steps = p->max_steps;
  T.flags = p->flags;
  for (int k = 0; k < 3; ++k) {
    T.light[k] = p->light_pos[k];
    T.background[k] = p->background[k];
  }
  T.light_intensity = p->light_intensity;
  T.eps_rel = p->eps_rel;
  T.ambient = p->ambient;
  T.out = (float4*)out_rgba;
  T.aov = out_aov;
  // scenes without sphere tracing whose trees are shallow enough for the
  // short stack take the analytic kernel (same arithmetic, fewer registers)
  T.ahs_march = s->L.ahs_march;
  T.analytic_small = s->L.analytic_only && s->L.stack_bound <= (uint32_t)kShortStackDepth && !T.S.tlas4 &&
                     !T.S.tlas8;
  T.counter = (unsigned long long*)counter;
  T.work = (unsigned long long*)work;
  s->trace_launches = launch_trace(T, st);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "trace launch");
  return PR_OK;
}

pr_status pr_trace(pr_scene* s, const pr_camera* camera, const pr_trace_params* params, float* out_rgba,
                   pr_aov* out_aov, uint64_t* ray_counter, void* stream) {
  if (!s || !camera || !out_rgba) return fail(PR_ERR_INVALID_ARG, "null scene/camera/output");
  if (!params_ok(params)) return PR_ERR_INVALID_ARG;
  if ((params->flags & PR_TRACE_WRITE_AOV) && !out_aov) return fail(PR_ERR_INVALID_ARG, "AOV requested but null");
  if (!s->built) return fail(PR_ERR_NOT_BUILT, "pr_trace before pr_build_bvh");
  return trace_impl(s, camera, nullptr, 1, params, out_rgba, out_aov, ray_counter, (cudaStream_t)stream);
}

// Camera frames of a multi-frame launch: computed here, copied to the scene's
// device array on the launch's stream.
static pr_status upload_frames(pr_scene* s, const pr_camera* cameras, uint32_t n_frames, const pr_trace_params* p,
                               cudaStream_t st) {
  if (s->cams_cap < n_frames) {
    if (s->d_frames) {
      cudaStreamSynchronize(st);
      cudaFree(s->d_frames);
      s->d_frames = nullptr;
      s->cams_cap = 0;
    }
    PR_CUDA(cudaMalloc(&s->d_frames, sizeof(CameraBasis) * n_frames), "cudaMalloc camera frames");
    s->cams_cap = n_frames;
  }
  s->h_frames.resize(n_frames);
  for (uint32_t f = 0; f < n_frames; ++f) s->h_frames[f] = camera_frame(cameras[f], p->width, p->height);
  PR_CUDA(cudaMemcpyAsync(s->d_frames, s->h_frames.data(), sizeof(CameraBasis) * n_frames, cudaMemcpyHostToDevice,
                          st),
          "copy camera frames");
  return PR_OK;
}

pr_status pr_trace_work(pr_scene* s, const pr_camera* cameras, uint32_t n_frames, const pr_trace_params* params,
                        float* out_rgba, uint64_t* work_counters, void* stream) {
  if (!s || !cameras || !out_rgba || !work_counters || n_frames == 0 || n_frames > 65535)
    return fail(PR_ERR_INVALID_ARG, "null scene/cameras/output/counters or n_frames outside 1..65535");
  if (!params_ok(params)) return PR_ERR_INVALID_ARG;
  if (!s->built) return fail(PR_ERR_NOT_BUILT, "pr_trace_work before pr_build_bvh");
  pr_trace_params q = *params;
  q.flags &= ~PR_TRACE_WRITE_AOV;
  cudaStream_t st = (cudaStream_t)stream;
  pr_status u = upload_frames(s, cameras, n_frames, &q, st);
  if (u != PR_OK) return u;
  return trace_impl(s, cameras, s->d_frames, n_frames, &q, out_rgba, nullptr, nullptr, st, work_counters);
}

pr_status pr_trace_frames(pr_scene* s, const pr_camera* cameras, uint32_t n_frames, const pr_trace_params* params,
                          float* out_rgba, pr_aov* out_aov, uint64_t* ray_counter, void* stream) {
  if (!s || !cameras || !out_rgba || n_frames == 0 || n_frames > 65535)
    return fail(PR_ERR_INVALID_ARG, "null scene/cameras/output or n_frames outside 1..65535");
  if (!params_ok(params)) return PR_ERR_INVALID_ARG;
  if ((params->flags & PR_TRACE_WRITE_AOV) && !out_aov) return fail(PR_ERR_INVALID_ARG, "AOV requested but null");
  if (!s->built) return fail(PR_ERR_NOT_BUILT, "pr_trace_frames before pr_build_bvh");
  cudaStream_t st = (cudaStream_t)stream;
  pr_status u = upload_frames(s, cameras, n_frames, params, st);
  if (u != PR_OK) return u;
  return trace_impl(s, cameras, s->d_frames, n_frames, params, out_rgba, out_aov, ray_counter, st);
}

pr_status pr_scene_error(pr_scene* s, void* stream, uint32_t* error_word) {
  if (!s || !error_word) return fail(PR_ERR_INVALID_ARG, "null scene/output");
  cudaStream_t st = (cudaStream_t)stream;
  uint32_t w = 0;
  PR_CUDA(cudaMemcpyAsync(&w, s->error_word, sizeof(w), cudaMemcpyDeviceToHost, st), "read error word");
  PR_CUDA(cudaMemsetAsync(s->error_word, 0, sizeof(uint32_t), st), "clear error word");
  PR_CUDA(cudaStreamSynchronize(st), "sync error word");
  *error_word = w;
  return PR_OK;
}

pr_status pr_scene_bounds(pr_scene* s, void* stream, float box[6]) {
  if (!s || !box) return fail(PR_ERR_INVALID_ARG, "null scene/output");
  if (!s->built) return fail(PR_ERR_NOT_BUILT, "scene not built");
  float b[8];
  cudaStream_t st = (cudaStream_t)stream;
  PR_CUDA(cudaMemcpyAsync(b, s->scene_box, sizeof(b), cudaMemcpyDeviceToHost, st), "read scene box");
  PR_CUDA(cudaStreamSynchronize(st), "sync scene box");
  box[0] = b[0]; box[1] = b[1]; box[2] = b[2]; box[3] = b[4]; box[4] = b[5]; box[5] = b[6];
  return PR_OK;
}

pr_status pr_scene_read_bvh(pr_scene* s, uint32_t level, void* stream, uint32_t cap, uint32_t* n_leaves_out,
                            uint32_t* perm, uint32_t* codes, int32_t* child, float* cbox, float* root_box) {
  if (!s) return fail(PR_ERR_INVALID_ARG, "null scene");
  if (!s->built) return fail(PR_ERR_NOT_BUILT, "scene not built");
  cudaStream_t st = (cudaStream_t)stream;
  const LevelDesc* J;
  uint32_t base = 0;
  if (level == PR_NONE) {
    J = &s->tlas_job;
  } else {
    if (level >= s->L.n_blas) return fail(PR_ERR_INVALID_ARG, "BLAS index out of range");
    J = nullptr;
    for (const LevelDesc& x : s->small_jobs)
      if (x.root_box == (float*)(s->blas_box + 2 * (size_t)level)) J = &x;
    for (const LevelDesc& x : s->large_blas)
      if (x.root_box == (float*)(s->blas_box + 2 * (size_t)level)) J = &x;
    base = J->leaf_ref_base;
  }
  const uint32_t n = J->n;
  if (n_leaves_out) *n_leaves_out = n;
  if (!perm && !codes && !child && !cbox && !root_box) return PR_OK;   // size query
  if (n > cap) return fail(PR_ERR_INVALID_ARG, "capacity too small");
  if (n == 0) return PR_OK;
  if (perm) PR_CUDA(cudaMemcpyAsync(perm, J->perm, sizeof(uint32_t) * n, cudaMemcpyDeviceToHost, st), "read perm");
  if (codes) PR_CUDA(cudaMemcpyAsync(codes, J->codes, sizeof(uint32_t) * n, cudaMemcpyDeviceToHost, st), "read codes");
  std::vector<float4> nodes(4 * (size_t)(n - 1));
  if (n > 1)
    PR_CUDA(cudaMemcpyAsync(nodes.data(), J->nodes, sizeof(float4) * nodes.size(), cudaMemcpyDeviceToHost, st),
            "read nodes");
  float rb[8];
  PR_CUDA(cudaMemcpyAsync(rb, J->root_box, sizeof(rb), cudaMemcpyDeviceToHost, st), "read root box");
  PR_CUDA(cudaStreamSynchronize(st), "sync read bvh");
  for (uint32_t i = 0; i + 1 < n; ++i) {
    const float* f = reinterpret_cast<const float*>(&nodes[4 * (size_t)i]);
    if (cbox) memcpy(cbox + 12 * (size_t)i, f, 12 * sizeof(float));
    if (child) {
      for (int side = 0; side < 2; ++side) {
        int32_t ref;
        memcpy(&ref, f + 12 + side, sizeof(ref));
        if (ref < 0) ref = (int32_t)(kLeafBit | (((uint32_t)ref & 0x7FFFFFFFu) - base));   // base holds the kind bit
        child[2 * (size_t)i + side] = ref;
      }
    }
  }
  if (root_box) {
    root_box[0] = rb[0]; root_box[1] = rb[1]; root_box[2] = rb[2];
    root_box[3] = rb[4]; root_box[4] = rb[5]; root_box[5] = rb[6];
  }
  return PR_OK;
}

pr_status pr_scene_kernel_launches(const pr_scene* s, uint32_t* build_launches, uint32_t* trace_launches) {
  if (!s) return fail(PR_ERR_INVALID_ARG, "null scene");
  if (build_launches) *build_launches = (uint32_t)s->build_launches;
  if (trace_launches) *trace_launches = (uint32_t)s->trace_launches;
  return PR_OK;
}

pr_status pr_lbvh_build(const float* boxes, uint32_t n, float* nodes, uint32_t* perm, uint32_t* codes,
                        float* root_box, void* stream) {
  if (n == 0) return PR_OK;
  if (!boxes || !perm || !codes || !root_box || (n > 1 && !nodes))
    return fail(PR_ERR_INVALID_ARG, "pr_lbvh_build: null device pointer");
  if (n > (1u << 28)) return fail(PR_ERR_INVALID_ARG, "pr_lbvh_build: more than 2^28 boxes");
  if (((uintptr_t)nodes & 15) || ((uintptr_t)root_box & 15))
    return fail(PR_ERR_INVALID_ARG, "pr_lbvh_build: nodes and root_box must be 16-byte aligned");
  cudaStream_t st = (cudaStream_t)stream;
  LevelDesc J;
  J.boxes = boxes;
  J.gather = nullptr;
  J.n = n;
  J.leaf_ref_base = 0;
  J.nodes = reinterpret_cast<float4*>(nodes);
  J.perm = perm;
  J.codes = codes;
  J.root_box = root_box;
  if (n <= kSmallMax) {
    launch_build_small_one(J, st);
  } else {
    void* scratch = nullptr;
    PR_CUDA(cudaMallocAsync(&scratch, build_scratch_bytes(n), st), "cudaMallocAsync LBVH scratch");
    launch_build_large(J, carve_build_scratch(scratch, n), st);
    PR_CUDA(cudaFreeAsync(scratch, st), "cudaFreeAsync LBVH scratch");
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "pr_lbvh_build launch");
  return PR_OK;
}

size_t pr_scene_device_bytes(const pr_scene* s) { return s ? s->arena_bytes + sizeof(CameraBasis) * s->cams_cap : 0; }

void pr_scene_destroy(pr_scene* s) {
  if (!s) return;
  cudaDeviceSynchronize();
  if (s->arena) cudaFree(s->arena);
  if (s->d_frames) cudaFree(s->d_frames);
  if (s->h_stage) cudaFreeHost(s->h_stage);
  if (s->stage_done) cudaEventDestroy(s->stage_done);
  if (s->tlas8f) cudaFree(s->tlas8f);
  delete s;
}

}  // extern "C"
