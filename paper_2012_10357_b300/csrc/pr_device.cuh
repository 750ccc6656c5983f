// Device-side scene layout shared by the BVH builder and the trace kernels.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/proceduray.h"

namespace pr {

constexpr uint32_t kLeafBit = 0x80000000u;
constexpr uint32_t kTriBit = 0x40000000u;    // a BLAS leaf ref of a triangle (kLeafBit | kTriBit | leaf)
// BLAS root ref of a procedural BLAS of 2..kLoopMaxLeaves leaves: kLeafBit |
// kLoopBit | (leaves - 1) << 27 | first leaf; the traversal tests its leaf
// boxes in a loop instead of walking its tree.
constexpr uint32_t kLoopBit = 0x20000000u;
constexpr uint32_t kLoopMaxLeaves = 4;
constexpr int kStackDepth = (int)PR_STACK_DEPTH;
// Stack of the analytic kernel variant, for scenes whose stack bound fits
constexpr int kShortStackDepth = 8;
constexpr uint32_t kErrSbt = 1u << PR_ERR_SBT_INDEX;
constexpr uint32_t kErrStack = 1u << PR_ERR_STACK_OVERFLOW;
constexpr int kEmptySlot = 0x7FFFFFFF;   // unused child slot of a 4- or 8-wide node
// Wide TLAS node formats (see the collapse in bvh.cu).
enum WideFormat : int { kWide4 = 4, kWide8 = 8, kWide8Q = 9 };

// One 4-wide node = 128 bytes = 8 x float4, child boxes stored by coordinate
// so the four slab tests run on whole vectors:
//   lo.x[4], lo.y[4], lo.z[4], hi.x[4], hi.y[4], hi.z[4], refs[4] (int bits), unused
// Empty slots have lo = +inf, hi = -inf (never entered) and ref kEmptySlot.

// One BVH2 node = 64 bytes = 4 x float4, both children's boxes stored in the
// parent so a visit is one node fetch:
//   n0 = (L.lo.x, L.lo.y, L.lo.z, L.hi.x)
//   n1 = (L.hi.y, L.hi.z, R.lo.x, R.lo.y)
//   n2 = (R.lo.z, R.hi.x, R.hi.y, R.hi.z)
//   n3 = (left ref, right ref, 0, 0) as int bits; ref >= 0 internal node,
//        ref = kLeafBit | leaf otherwise.
struct BlasInfo {      // int4 on the device
  int node_base;       // first node of this BLAS in the BLAS node array
  int leaf_base;       // first entry of this BLAS in the flattened leaf arrays
  int n_leaves;
  int root_ref;        // 0 (node_base + 0), kLeafBit | leaf (single leaf), or a leaf loop (kLoopBit)
};

// Everything a trace kernel reads; passed by value.
struct SceneView {
  // instances (creation order): one 96-byte record each, read with six
  // independent 16-byte loads when a ray reaches the instance
  //   [0..2] world->object rows (linear xyz, translation w)
  //   [3]    BLAS root box lo.xyz, BLAS root ref (int bits)
  //   [4]    BLAS root box hi.xyz, BLAS first node (int bits)
  //   [5]    blas, sbt_offset, inst_id, mask (uint bits)
  const float4* inst_rec;
  // TLAS
  const float4* tlas_nodes;   // [max(n_inst-1,0)][4]
  int tlas_root_ref;          // 0 or kLeafBit | instance (single instance)
  const float4* tlas4;        // [n4][8] 4-wide TLAS collapsed from the binary one, or null
  int tlas4_root;             // 0 or kLeafBit | instance (root of the 4- or 8-wide TLAS)
  const float4* tlas8;        // 8-wide TLAS ([n8][14] float or [n8][6] quantised nodes), or null
  int tlas8_format;           // kWide8 or kWide8Q when tlas8 is set
  const float* scene_box;     // [6] TLAS root box (world)
  // BLAS
  const int4* blas_info;      // [n_blas] BlasInfo
  const float4* blas_box;     // [n_blas][2] object-space root box (lo.xyz,_),(hi.xyz,_)
  const float4* blas_nodes;   // [sum(n_leaves-1)][4]
  // flattened BLAS leaves (geometry-major per BLAS)
  const uint32_t* leaf_prim;  // global primitive index
  const uint2* leaf_gq;       // (g inside the BLAS, primitive index inside geometry)
  const float* vertices;      // [n_vertices][3] triangle vertices (object space)
  const uint32_t* indices;    // [n_triangles][3]
  // primitives
  const float* aabbs;         // [n_prims][6]
  const float4* params;       // [n_prims][4]
  // shader binding
  const uint4* sbt;           // [n_records] the record's hit group resolved: is, chs, ahs, material
  const float4* materials;    // [n_materials]
  const uint2* ray_types;     // [n_ray_types] miss, flags
  uint32_t n_inst, n_blas, n_records, sbt_stride_m;
  uint32_t* error_word;
};

// Pinhole camera frame of one image (ray generation, Section 2.2.3), as the
// kernels read it: the host computes it once per frame (camera_frame) and each
// thread forms its pixel's ray from it (camera_ray).
struct CameraBasis {
  float3 eye, fwd, right, up;
  float kx, ky;     // 2 / W, 2 / H
  float ax, ay;     // tan(fov/2) * aspect, -tan(fov/2)
};

}  // namespace pr
