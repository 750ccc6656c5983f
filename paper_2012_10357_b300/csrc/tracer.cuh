// Shared device-side tracing: traversal of the two-level BVH, Eq. 1 dispatch,
// surface reconstruction and shading arithmetic. Used by the megakernel
// (trace.cu) and by the batched wavefront kernels (wavefront.cu); the shading
// composition uses explicitly rounded operations so both produce the same bits.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "pr_device.cuh"
#include "shaders.cuh"

namespace pr {

#ifndef PR_WHILE_WHILE
#define PR_WHILE_WHILE 0
#endif
// While-while order in the 4-wide TLAS traversal (used from 64 instances up).
#ifndef PR_TLAS4_WHILE_WHILE
#define PR_TLAS4_WHILE_WHILE 0
#endif

// Per-thread traversal stack. With PR_SMEM_STACK (default) the entries live in
// shared memory, interleaved across the CTA's threads (entry i of thread t at
// i * blockDim + t, conflict-free): 32 KB per 128-thread CTA. Otherwise in a
// per-thread local array. Measured on B300 (interleaved A/B, same box):
// shared stack with 4 CTAs/SM is 8-25 % faster than the local array.
struct TravStack {
  int* p;
  int stride;
  __device__ __forceinline__ int& operator[](int i) const { return p[i * stride]; }
};

struct Hit {
  float t;
  int inst;        // instance index, -1 = none
  int leaf;        // flattened BLAS leaf
  uint32_t attr;   // intersection attribute
};

// Fractal march candidates a traversal hands on instead of marching them in
// place (the regrouped wavefront runs them later from a job queue): the
// instance, the leaf, the record's shader and primitive, and the leaf's slab
// interval. Beyond kMaxDeferred candidates a ray marches in place.
constexpr int kMaxDeferred = 4;
struct Deferred {
  int n;
  int inst[kMaxDeferred], leaf[kMaxDeferred];
  uint32_t is_id[kMaxDeferred], prim[kMaxDeferred];
  float t_lo[kMaxDeferred], t_hi[kMaxDeferred];
  float3 oo[kMaxDeferred], dd[kMaxDeferred];   // the ray in the instance's object space
};

__device__ __forceinline__ bool is_fractal(uint32_t id) {
  return id == PR_IS_JULIA || id == PR_IS_MANDELBULB || id == PR_IS_JULIA_CUT;
}

__device__ __forceinline__ bool key_less(int i0, uint2 gq0, int i1, uint2 gq1) {
  if (i0 != i1) return i0 < i1;
  if (gq0.x != gq1.x) return gq0.x < gq1.x;
  return gq0.y < gq1.y;
}

__device__ __forceinline__ void node_boxes(const float4* n, float3 inv_d, float3 o_inv, float tmin, float tmax,
                                           float& l0, float& l1, float& r0, float& r1, int& lref, int& rref) {
  float4 a = __ldg(n), b = __ldg(n + 1), c = __ldg(n + 2), e = __ldg(n + 3);
  slab_clip(f3(a.x, a.y, a.z), f3(a.w, b.x, b.y), inv_d, o_inv, tmin, tmax, l0, l1);
  slab_clip(f3(b.z, b.w, c.x), f3(c.y, c.z, c.w), inv_d, o_inv, tmin, tmax, r0, r1);
  lref = __float_as_int(e.x);
  rref = __float_as_int(e.y);
}

// Intersection shader dispatch on the hit group's shader id (kAnalytic: the
// scene has no sphere-traced shader, so that code is not compiled in).
template <bool kAnalytic, bool kAhs = false, bool kInlineMarch = false>
__device__ __forceinline__ bool run_intersection(uint32_t is_id, uint32_t ahs, const float4* prm, float3 o, float3 d,
                                                 float3 inv_d, float tmin, float t_lo, float t_hi, float eps,
                                                 uint32_t max_steps, IsResult& r, WorkCounters* wc) {
  if (wc) ++wc->is_calls[is_id < PR_IS_COUNT ? is_id : 0];
  switch (is_id) {
    case PR_IS_SPHERE: return is_sphere(__ldg(prm), o, d, tmin, r, ahs);
    case PR_IS_BOX: return is_box(__ldg(prm), __ldg(prm + 1), o, d, inv_d, tmin, r, ahs);
    case PR_IS_PACMAN: return is_pacman(__ldg(prm), __ldg(prm + 1), o, d, tmin, r, ahs);
    default:
      if (!kAnalytic && is_sphere_traced(is_id)) {
        const float inv_len = rsqrtf(dot3(d, d));
        auto march = [&](float t0, uint32_t steps) {
          if constexpr (kInlineMarch) return sphere_trace_body(is_id, prm, o, d, inv_len, t0, t_hi, eps, steps, wc);
          else return sphere_trace(is_id, prm, o, d, inv_len, t0, t_hi, eps, steps, wc);
        };
        r = march(t_lo, max_steps);
        if constexpr (kAhs) {
          // Every march point below eps is a candidate for the any-hit shader; an
          // ignored one lets the march go on by max(|estimate|, eps), through the
          // solid and out of it, within the same step budget. (Compiled only into
          // the kernels of scenes that need it: the extra call site costs the
          // others 6-10 %.)
          uint32_t used = 0;
          while (ahs != PR_NONE && r.attr != 0u && !any_hit_accepts(ahs, o, r.t, d)) {
            used += r.attr;
            if (used >= max_steps) {
              r.attr = 0u;
              break;
            }
            r = march(r.t + fmaxf(fabsf(r.dist), eps), max_steps - used);
          }
          if (r.attr != 0u) r.attr += used;
        }
        return r.attr != 0u;
      }
      return false;
  }
}

__device__ __forceinline__ void to_object(float4 m0, float4 m1, float4 m2, float3 o, float3 d, float3& oo, float3& dd) {
  oo = f3(fmaf(m0.x, o.x, fmaf(m0.y, o.y, fmaf(m0.z, o.z, m0.w))), fmaf(m1.x, o.x, fmaf(m1.y, o.y, fmaf(m1.z, o.z, m1.w))),
          fmaf(m2.x, o.x, fmaf(m2.y, o.y, fmaf(m2.z, o.z, m2.w))));
  dd = f3(fmaf(m0.x, d.x, fmaf(m0.y, d.y, m0.z * d.z)), fmaf(m1.x, d.x, fmaf(m1.y, d.y, m1.z * d.z)),
          fmaf(m2.x, d.x, fmaf(m2.y, d.y, m2.z * d.z)));
}

// BLAS traversal of instance k (object-space ray; t shared with world space
// because the direction is not renormalised). Returns true if any-hit mode
// found a hit.
template <bool kStats, bool kAnalytic = false, int kDepth = kStackDepth, bool kDefer = false, bool kAhs = false,
          bool kInlineMarch = false>
__device__ bool traverse_blas(bool any_hit, const SceneView& S, int k, float3 o, float3 d, uint32_t r, float tmin, float eps,
                              uint32_t max_steps, Hit& h, TravStack stack, int sp0, WorkCounters* wc_,
                              Deferred* defer = nullptr) {
  WorkCounters* wc = kStats ? wc_ : nullptr;
  if (wc) ++wc->instances;
  const float4* R = S.inst_rec + 6 * (size_t)k;
  const float4 m0 = __ldg(R), m1 = __ldg(R + 1), m2 = __ldg(R + 2), blo = __ldg(R + 3), bhi = __ldg(R + 4);
  const uint4 info = __ldg(reinterpret_cast<const uint4*>(R + 5));   // blas, sbt_offset, inst_id, mask
  if ((info.w & 0xFFu) == 0u) return false;
  float3 oo, dd;
  to_object(m0, m1, m2, o, d, oo, dd);
  float3 inv = safe_rcp(dd);
  float3 o_inv = f3(-oo.x * inv.x, -oo.y * inv.y, -oo.z * inv.z);
  const int root_ref = __float_as_int(blo.w), node_base = __float_as_int(bhi.w);
  float r_lo, r_hi;   // root-box slab interval
  slab_clip(f3(blo.x, blo.y, blo.z), f3(bhi.x, bhi.y, bhi.z), inv, o_inv, tmin, h.t, r_lo, r_hi);
  if (r_lo > r_hi) return false;
  // Slab interval of a primitive's AABB (lo.xyz, hi.xyz) clipped to [tmin,
  // h.t]: the entry and exit plane of each axis are picked once per ray by the
  // sign of 1/d (an FMA is monotone in the plane, so the picked plane gives
  // exactly the min / max of the axis's two slab distances) and only those
  // words are read, with no min / max per axis.
  const int pnx = inv.x >= 0.f ? 0 : 3, pny = inv.y >= 0.f ? 1 : 4, pnz = inv.z >= 0.f ? 2 : 5;
  auto leaf_slab = [&](const float* bb, float& t_lo, float& t_hi) {
    t_lo = fmax3(fmaf(__ldg(bb + pnx), inv.x, o_inv.x), fmaf(__ldg(bb + pny), inv.y, o_inv.y),
                 fmaxf(fmaf(__ldg(bb + pnz), inv.z, o_inv.z), tmin));
    t_hi = fmin3(fmaf(__ldg(bb + (3 - pnx)), inv.x, o_inv.x), fmaf(__ldg(bb + (5 - pny)), inv.y, o_inv.y),
                 fminf(fmaf(__ldg(bb + (7 - pnz)), inv.z, o_inv.z), h.t));
  };
  // Procedural leaf whose AABB slab interval is [t_lo, t_hi]: Eq. 1 record,
  // intersection shader, closest-hit bookkeeping. True when any-hit mode
  // accepted a hit (the trace ends).
  auto procedural_leaf = [&](int leaf, uint32_t prim, float t_lo, float t_hi) -> bool {
    uint2 gq = __ldg(S.leaf_gq + leaf);
    if (wc) ++wc->sbt_lookups;
    uint32_t rec = r + S.sbt_stride_m * gq.x + info.y;
    if (rec >= S.n_records) {
      atomicOr(S.error_word, kErrSbt);
      return false;
    }
    const uint4 hg = __ldg(S.sbt + rec);   // is, chs, ahs, material
    if (kDefer && is_fractal(hg.x) && hg.z == PR_NONE && defer->n < kMaxDeferred) {   // any-hit candidates march here
      const int i = defer->n++;
      defer->inst[i] = k;
      defer->leaf[i] = leaf;
      defer->is_id[i] = hg.x;
      defer->prim[i] = prim;
      defer->t_lo[i] = t_lo;
      defer->t_hi[i] = t_hi;
      defer->oo[i] = oo;
      defer->dd[i] = dd;
      return false;
    }
    IsResult res;
    if (run_intersection<kAnalytic, kAhs, kInlineMarch>(hg.x, hg.z, S.params + 4 * (size_t)prim, oo, dd, inv, tmin, t_lo, t_hi, eps, max_steps, res, wc) &&
        res.t >= tmin) {
      bool accept = res.t < h.t;
      if (!accept && res.t == h.t && h.inst >= 0)
        accept = key_less(k, gq, h.inst, __ldg(S.leaf_gq + (h.leaf & 0x3FFFFFFF)));
      if (accept) {
        h.t = res.t;
        h.inst = k;
        h.leaf = leaf;
        h.attr = res.attr;
        if (any_hit) return true;
      }
    }
    return false;
  };
  if constexpr (kAnalytic) {
    if (root_ref < 0 && (root_ref & (int)kLoopBit)) {
    // Procedural BLAS of 2..4 leaves: every leaf box is tested in turn. The
    // tree's node tests are the same slab tests on the same boxes with a stack
    // around them, and the closest hit does not depend on the order in which
    // the leaves are met (ties go by key), so the result is the tree's.
    // (Only in the analytic kernel variant: compiled into the generic kernel,
    // the loop cost its other paths 4-8 % through register allocation.)
    const int first = root_ref & 0x07FFFFFF, cnt = ((root_ref >> 27) & 3) + 1;
    for (int j = 0; j < cnt; ++j) {
      const int leaf = first + j;
      if (wc) ++wc->leaves;
      const uint32_t prim = __ldg(S.leaf_prim + leaf);
      // the box as three 8-byte words (24-byte records, 8-byte aligned)
      const float2* bb = reinterpret_cast<const float2*>(S.aabbs + 6 * (size_t)prim);
      const float2 u = __ldg(bb), v = __ldg(bb + 1), w = __ldg(bb + 2);
      float t_lo, t_hi;
      slab_clip(f3(u.x, u.y, v.x), f3(v.y, w.x, w.y), inv, o_inv, tmin, h.t, t_lo, t_hi);
      if (t_lo <= t_hi && procedural_leaf(leaf, prim, t_lo, t_hi)) return true;
    }
    return false;
    }
  }
  if (root_ref < 0 && !(root_ref & (int)kTriBit) && !(root_ref & (int)kLoopBit)) {
    // One-AABB BLAS: the build copies that AABB as the root box, so the root
    // slab interval is the leaf's own; no second slab test.
    const int leaf = root_ref & 0x3FFFFFFF;
    return procedural_leaf(leaf, __ldg(S.leaf_prim + leaf), r_lo, r_hi);
  }
  int sp = sp0;
  // a leaf-loop BLAS (kLoopBit; leaf refs stay below 2^29) walks its tree here
  int node = (root_ref < 0 && (root_ref & (int)kLoopBit)) ? 0 : root_ref;
  for (;;) {
    if (node >= 0) {
      float l0, l1, r0, r1;
      int lref, rref;
      if (wc) ++wc->blas_nodes;
      node_boxes(S.blas_nodes + 4 * (size_t)(node_base + node), inv, o_inv, tmin, h.t, l0, l1, r0, r1, lref, rref);
      bool hl = l0 <= l1, hr = r0 <= r1;
      if (hl && hr) {
        int nearr = lref, farr = rref;
        if (r0 < l0) { nearr = rref; farr = lref; }
        if (sp < kDepth) stack[sp++] = farr;
        else atomicOr(S.error_word, kErrStack);
        node = nearr;
        continue;
      }
      if (hl) { node = lref; continue; }
      if (hr) { node = rref; continue; }
    } else {
      const bool tri = (node & (int)kTriBit) != 0;
      int leaf = node & 0x3FFFFFFF;
      if (wc) ++wc->leaves;
      uint32_t prim = __ldg(S.leaf_prim + leaf);
      if (tri) {
        // built-in triangle intersection; the record supplies the hit group (any-hit shader)
        uint2 gq = __ldg(S.leaf_gq + leaf);
        uint32_t rec = r + S.sbt_stride_m * gq.x + info.y;
        if (rec >= S.n_records) {
          atomicOr(S.error_word, kErrSbt);
        } else {
          const uint32_t ahs = __ldg(S.sbt + rec).z;
          const uint32_t* ti = S.indices + 3 * (size_t)prim;
          float t;
          const float3 v0 = ldf3g(S.vertices + 3 * (size_t)__ldg(ti));
          const float3 v1 = ldf3g(S.vertices + 3 * (size_t)__ldg(ti + 1));
          const float3 v2 = ldf3g(S.vertices + 3 * (size_t)__ldg(ti + 2));
          if (is_triangle(v0, v1, v2, oo, dd, tmin, t, ahs)) {
            bool accept = t < h.t;
            if (!accept && t == h.t && h.inst >= 0)
              accept = key_less(k, gq, h.inst, __ldg(S.leaf_gq + (h.leaf & 0x3FFFFFFF)));
            if (accept) {
              h.t = t;
              h.inst = k;
              h.leaf = leaf | (int)kTriBit;
              h.attr = 0;
              if (any_hit) return true;
            }
          }
        }
        if (sp == sp0) break;
        node = stack[--sp];
        continue;
      }
      float t_lo, t_hi;
      leaf_slab(S.aabbs + 6 * (size_t)prim, t_lo, t_hi);
      if (t_lo <= t_hi && procedural_leaf(leaf, prim, t_lo, t_hi)) return true;
    }
    if (sp == sp0) break;
    node = stack[--sp];
  }
  return false;
}

// One TraceRay: TLAS traversal (near child first), instance transition, BLAS.
// kTlas: 0 = the 4-wide TLAS when the scene has one, else the binary one;
// kWide8 / kWide8Q = the scene's 8-wide TLAS (float / quantised nodes).
template <bool kStats, bool kAnalytic = false, int kDepth = kStackDepth, bool kDefer = false, int kTlas = 0,
          bool kAhs = false, bool kInlineMarch = false>
__device__ __forceinline__ void trace_ray_body(bool any_hit, const SceneView& S, float3 o, float3 d, uint32_t r, float tmin,
                                               float tmax, float eps, uint32_t max_steps, Hit& h, TravStack stack,
                                               WorkCounters* wc_, Deferred* defer) {
  WorkCounters* wc = kStats ? wc_ : nullptr;
  if (wc) ++wc->rays;
  h.t = tmax;
  h.inst = -1;
  h.leaf = -1;
  h.attr = 0;
  if (S.n_inst == 0) return;
  float3 inv = safe_rcp(d);
  float3 o_inv = f3(-o.x * inv.x, -o.y * inv.y, -o.z * inv.z);
  int sp = 0;
  if constexpr (kTlas == kWide8 || kTlas == kWide8Q) {
    // 8-wide TLAS: eight slab tests per node, hit children ordered near to far
    // by a 19-exchange sorting network (Batcher's odd-even merge sort); the
    // nearest is visited next, the others pushed farthest first. Quantised
    // nodes decode a bound as origin + q * 2^e inside the slab test: with
    // a = 2^e / d and b = (origin - o) / d, t = q * a + b, and the entry
    // and exit bounds of each axis are picked once per node by the sign of d.
    constexpr int kNone = 0x7FFFFFFF;
    const bool px = inv.x >= 0.f, py = inv.y >= 0.f, pz = inv.z >= 0.f;
    auto visit8 = [&](int node) -> int {
      if (wc) ++(kTlas == kWide8Q ? wc->tlas_nodes8q : wc->tlas_nodes8);
      float key[8];
      int ref[8];
      if constexpr (kTlas == kWide8Q) {
        const float4* nd = S.tlas8 + 6 * (size_t)node;
        const float4 h0 = __ldg(nd);
        const float4 fx = __ldg(nd + 1), fy = __ldg(nd + 2), fz = __ldg(nd + 3);
        const int4 r0 = __ldg(reinterpret_cast<const int4*>(nd + 4)), r1 = __ldg(reinterpret_cast<const int4*>(nd + 5));
        ref[0] = r0.x; ref[1] = r0.y; ref[2] = r0.z; ref[3] = r0.w;
        ref[4] = r1.x; ref[5] = r1.y; ref[6] = r1.z; ref[7] = r1.w;
        const uint32_t eb = __float_as_uint(h0.w);
        const float ax = __uint_as_float((eb & 0xFFu) << 23) * inv.x;
        const float ay = __uint_as_float(((eb >> 8) & 0xFFu) << 23) * inv.y;
        const float az = __uint_as_float(((eb >> 16) & 0xFFu) << 23) * inv.z;
        const float bx = fmaf(h0.x, inv.x, o_inv.x), by = fmaf(h0.y, inv.y, o_inv.y), bz = fmaf(h0.z, inv.z, o_inv.z);
        // entry (n) and exit (f) byte words per axis: {children 0-3, 4-7}
        const uint32_t wx[4] = {__float_as_uint(fx.x), __float_as_uint(fx.y), __float_as_uint(fx.z), __float_as_uint(fx.w)};
        const uint32_t wy[4] = {__float_as_uint(fy.x), __float_as_uint(fy.y), __float_as_uint(fy.z), __float_as_uint(fy.w)};
        const uint32_t wz[4] = {__float_as_uint(fz.x), __float_as_uint(fz.y), __float_as_uint(fz.z), __float_as_uint(fz.w)};
        const uint32_t nx[2] = {px ? wx[0] : wx[2], px ? wx[1] : wx[3]}, fxw[2] = {px ? wx[2] : wx[0], px ? wx[3] : wx[1]};
        const uint32_t ny[2] = {py ? wy[0] : wy[2], py ? wy[1] : wy[3]}, fyw[2] = {py ? wy[2] : wy[0], py ? wy[3] : wy[1]};
        const uint32_t nz[2] = {pz ? wz[0] : wz[2], pz ? wz[1] : wz[3]}, fzw[2] = {pz ? wz[2] : wz[0], pz ? wz[3] : wz[1]};
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          // byte k of a word as a float: 2^23 + q (exponent byte 0x4B), minus 2^23
          const uint32_t sel = 0x7540u | (uint32_t)(k & 3);
          auto dq = [&](uint32_t w) { return __uint_as_float(__byte_perm(w, 0x4B000000u, sel)) - 8388608.f; };
          const float tnx = fmaf(dq(nx[k >> 2]), ax, bx), tfx = fmaf(dq(fxw[k >> 2]), ax, bx);
          const float tny = fmaf(dq(ny[k >> 2]), ay, by), tfy = fmaf(dq(fyw[k >> 2]), ay, by);
          const float tnz = fmaf(dq(nz[k >> 2]), az, bz), tfz = fmaf(dq(fzw[k >> 2]), az, bz);
          const float t0 = fmax3(tnx, tny, fmaxf(tnz, tmin));
          const float t1 = fmin3(tfx, tfy, fminf(tfz, h.t));
          key[k] = (ref[k] != kEmptySlot && t0 <= t1) ? t0 : INFINITY;
        }
      } else {
        const float4* nd = S.tlas8 + 14 * (size_t)node;
        float4 v[14];
#pragma unroll
        for (int q = 0; q < 14; ++q) v[q] = __ldg(nd + q);
        const float* f = reinterpret_cast<const float*>(v);
#pragma unroll
        for (int k = 0; k < 8; ++k) ref[k] = __float_as_int(f[48 + k]);
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          const float ax = fmaf(f[k], inv.x, o_inv.x), bx = fmaf(f[24 + k], inv.x, o_inv.x);
          const float ay = fmaf(f[8 + k], inv.y, o_inv.y), by = fmaf(f[32 + k], inv.y, o_inv.y);
          const float az = fmaf(f[16 + k], inv.z, o_inv.z), bz = fmaf(f[40 + k], inv.z, o_inv.z);
          const float t0 = fmax3(fminf(ax, bx), fminf(ay, by), fmaxf(fminf(az, bz), tmin));
          const float t1 = fmin3(fmaxf(ax, bx), fmaxf(ay, by), fminf(fmaxf(az, bz), h.t));
          key[k] = (ref[k] != kEmptySlot && t0 <= t1) ? t0 : INFINITY;
        }
      }
      auto cswap = [&](int a, int b) {
        if (key[b] < key[a]) {
          float tk = key[a]; key[a] = key[b]; key[b] = tk;
          int tr = ref[a]; ref[a] = ref[b]; ref[b] = tr;
        }
      };
      cswap(0, 1); cswap(2, 3); cswap(4, 5); cswap(6, 7);
      cswap(0, 2); cswap(1, 3); cswap(4, 6); cswap(5, 7);
      cswap(1, 2); cswap(5, 6);
      cswap(0, 4); cswap(1, 5); cswap(2, 6); cswap(3, 7);
      cswap(2, 4); cswap(3, 5);
      cswap(1, 2); cswap(3, 4); cswap(5, 6);
      if (key[0] == INFINITY) return kNone;
#pragma unroll
      for (int k = 7; k >= 1; --k) {
        if (key[k] != INFINITY) {
          if (sp < kDepth) stack[sp++] = ref[k];
          else atomicOr(S.error_word, kErrStack);
        }
      }
      return ref[0];
    };
    int node = S.tlas4_root;   // 0 or kLeafBit | instance
    for (;;) {
      if (node >= 0) {
        node = visit8(node);
        if (node != kNone) continue;
      } else if (traverse_blas<kStats, kAnalytic, kDepth, kDefer, kAhs, kInlineMarch>(any_hit, S, node & 0x7FFFFFFF, o, d, r, tmin, eps, max_steps, h, stack, sp, wc, defer)) {
        return;
      }
      if (sp == 0) return;
      node = stack[--sp];
    }
  }
  if (S.tlas4) {
    // 4-wide TLAS: four slab tests per node on coordinate vectors, hit
    // children ordered near to far by a 5-exchange sorting network; the
    // nearest is visited next, the others pushed farthest first.
    constexpr int kNone = 0x7FFFFFFF;   // no node (never a node index: those are < 2^30)
    // Entry and exit planes per axis by the sign of d (rows lo.x, lo.y, lo.z,
    // hi.x, hi.y, hi.z of a node): an FMA is monotone in the plane, so the
    // plane picked by the sign gives exactly min / max of the two slab
    // distances (empty slots are masked by their ref) and the node's rows are
    // read in that order, with no min / max per axis.
    const int rnx = inv.x >= 0.f ? 0 : 3, rny = inv.y >= 0.f ? 1 : 4, rnz = inv.z >= 0.f ? 2 : 5;
    auto visit4 = [&](int node) -> int {
      if (wc) ++wc->tlas_nodes4;
      const float4* nd = S.tlas4 + 8 * (size_t)node;
      const float4 nx = __ldg(nd + rnx), ny = __ldg(nd + rny), nz = __ldg(nd + rnz);
      const float4 fx = __ldg(nd + (3 - rnx)), fy = __ldg(nd + (5 - rny)), fz = __ldg(nd + (7 - rnz)),
                   rf = __ldg(nd + 6);
      const float cn[3][4] = {{nx.x, nx.y, nx.z, nx.w}, {ny.x, ny.y, ny.z, ny.w}, {nz.x, nz.y, nz.z, nz.w}};
      const float cf[3][4] = {{fx.x, fx.y, fx.z, fx.w}, {fy.x, fy.y, fy.z, fy.w}, {fz.x, fz.y, fz.z, fz.w}};
      int ref[4] = {__float_as_int(rf.x), __float_as_int(rf.y), __float_as_int(rf.z), __float_as_int(rf.w)};
      float key[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const float t0 = fmax3(fmaf(cn[0][k], inv.x, o_inv.x), fmaf(cn[1][k], inv.y, o_inv.y),
                               fmaxf(fmaf(cn[2][k], inv.z, o_inv.z), tmin));
        const float t1 = fmin3(fmaf(cf[0][k], inv.x, o_inv.x), fmaf(cf[1][k], inv.y, o_inv.y),
                               fminf(fmaf(cf[2][k], inv.z, o_inv.z), h.t));
        key[k] = (ref[k] != kEmptySlot && t0 <= t1) ? t0 : INFINITY;
      }
      auto cswap = [&](int a, int b) {
        if (key[b] < key[a]) {
          float tk = key[a]; key[a] = key[b]; key[b] = tk;
          int tr = ref[a]; ref[a] = ref[b]; ref[b] = tr;
        }
      };
      cswap(0, 1); cswap(2, 3); cswap(0, 2); cswap(1, 3); cswap(1, 2);
      if (key[0] == INFINITY) return kNone;
#pragma unroll
      for (int k = 3; k >= 1; --k) {
        if (key[k] != INFINITY) {
          if (sp < kDepth) stack[sp++] = ref[k];
          else atomicOr(S.error_word, kErrStack);
        }
      }
      return ref[0];
    };
    int node = S.tlas4_root;
#if PR_TLAS4_WHILE_WHILE
    // While-while order (Aila & Laine 2009): descend until every converged
    // lane of the warp holds an instance leaf (or is done), then run the
    // instance transitions and BLAS work of the warp together.
    while (node != kNone) {
      int leaf = kNone;
      while (node != kNone) {
        if (node >= 0) {
          node = visit4(node);
          if (node == kNone) node = sp ? stack[--sp] : kNone;
        }
        if (node < 0) {
          if (leaf != kNone) break;   // already holding one: go process it
          leaf = node;
          node = sp ? stack[--sp] : kNone;
        }
        if (!__any_sync(__activemask(), leaf == kNone)) break;
      }
      if (leaf != kNone &&
          traverse_blas<kStats, kAnalytic, kDepth, kDefer, kAhs, kInlineMarch>(any_hit, S, leaf & 0x7FFFFFFF, o, d, r, tmin, eps, max_steps, h, stack, sp, wc, defer))
        return;
    }
    return;
#else
    for (;;) {
      if (node >= 0) {
        node = visit4(node);
        if (node != kNone) continue;
      } else if (traverse_blas<kStats, kAnalytic, kDepth, kDefer, kAhs, kInlineMarch>(any_hit, S, node & 0x7FFFFFFF, o, d, r, tmin, eps, max_steps, h, stack, sp, wc, defer)) {
        return;
      }
      if (sp == 0) return;
      node = stack[--sp];
    }
#endif
  }
  int node = S.tlas_root_ref;
#if PR_WHILE_WHILE
  // While-while traversal (Aila & Laine 2009): descend internal nodes, hold
  // back the first instance leaf reached and keep descending until every
  // converged lane of the warp holds a leaf (or is done), then run the
  // instance transitions and BLAS work together.
  constexpr int kDone = 0x7FFFFFFF;
  while (node != kDone) {
    int leaf = kDone;
    while (node != kDone) {
      if (node >= 0) {
        float l0, l1, r0, r1;
        int lref, rref;
        if (wc) ++wc->tlas_nodes;
        node_boxes(S.tlas_nodes + 4 * (size_t)node, inv, o_inv, tmin, h.t, l0, l1, r0, r1, lref, rref);
        const bool hl = l0 <= l1, hr = r0 <= r1;
        if (hl && hr) {
          int nearr = lref, farr = rref;
          if (r0 < l0) { nearr = rref; farr = lref; }
          if (sp < kDepth) stack[sp++] = farr;
          else atomicOr(S.error_word, kErrStack);
          node = nearr;
        } else if (hl) {
          node = lref;
        } else if (hr) {
          node = rref;
        } else {
          node = sp ? stack[--sp] : kDone;
        }
      }
      if (node < 0) {
        if (leaf != kDone) break;          // already holding a leaf: go process it
        leaf = node;
        node = sp ? stack[--sp] : kDone;
      }
      if (!__any_sync(__activemask(), leaf == kDone)) break;
    }
    if (leaf != kDone &&
        traverse_blas<kStats, kAnalytic, kDepth, kDefer, kAhs, kInlineMarch>(any_hit, S, leaf & 0x7FFFFFFF, o, d, r, tmin, eps, max_steps, h, stack, sp, wc, defer))
      return;
  }
#else
  for (;;) {
    if (node >= 0) {
      float l0, l1, r0, r1;
      int lref, rref;
      if (wc) ++wc->tlas_nodes;
      node_boxes(S.tlas_nodes + 4 * (size_t)node, inv, o_inv, tmin, h.t, l0, l1, r0, r1, lref, rref);
      bool hl = l0 <= l1, hr = r0 <= r1;
      if (hl && hr) {
        int nearr = lref, farr = rref;
        if (r0 < l0) { nearr = rref; farr = lref; }
        if (sp < kDepth) stack[sp++] = farr;
        else atomicOr(S.error_word, kErrStack);
        node = nearr;
        continue;
      }
      if (hl) { node = lref; continue; }
      if (hr) { node = rref; continue; }
    } else {
      if (traverse_blas<kStats, kAnalytic, kDepth, kDefer, kAhs, kInlineMarch>(any_hit, S, node & 0x7FFFFFFF, o, d, r, tmin, eps, max_steps, h, stack, sp, wc, defer)) return;
    }
    if (sp == 0) break;
    node = stack[--sp];
  }
#endif
}

// Out of line: one copy of the traversal serves every call site (the
// instruction cache holds the megakernel's working set). The hit comes back
// by value, in registers, not through the caller's stack frame.
template <bool kStats, bool kAnalytic = false, int kDepth = kStackDepth, bool kDefer = false, int kTlas = 0,
          bool kAhs = false, bool kInlineMarch = false>
__device__ __noinline__ Hit trace_ray(bool any_hit, const SceneView& S, float3 o, float3 d, uint32_t r, float tmin,
                                      float tmax, float eps, uint32_t max_steps, TravStack stack, WorkCounters* wc,
                                      Deferred* defer) {
  Hit h;
  trace_ray_body<kStats, kAnalytic, kDepth, kDefer, kTlas, kAhs, kInlineMarch>(any_hit, S, o, d, r, tmin, tmax, eps,
                                                                               max_steps, h, stack, wc, defer);
  return h;
}

// The analytic kernel (no estimators: a small instruction footprint) takes
// the traversal inline, at one site (render_pixel_one_site): no call's
// register saves (4096 64x64 frames: 32.0 Grays/s through the call, 34.0
// inline at each ray's site, 38.6 at one site). The generic kernel keeps it
// out of line.
#ifndef PR_ANALYTIC_INLINE
#define PR_ANALYTIC_INLINE 1
#endif

template <bool kStats, bool kAnalytic = false, int kDepth = kStackDepth, bool kDefer = false, int kTlas = 0,
          bool kAhs = false, bool kInlineMarch = false>
__device__ __forceinline__ void trace_typed(const SceneView& S, float3 o, float3 d, uint32_t r, float tmin, float tmax,
                                            float eps, uint32_t max_steps, Hit& h, TravStack stack, WorkCounters* wc,
                                            Deferred* defer = nullptr) {
  const bool any_hit = (__ldg(S.ray_types + r).y & PR_RAY_TERMINATE_ON_FIRST_HIT) != 0;
  if constexpr (kAnalytic && PR_ANALYTIC_INLINE)
    trace_ray_body<kStats, kAnalytic, kDepth, kDefer, kTlas, kAhs, kInlineMarch>(any_hit, S, o, d, r, tmin, tmax, eps, max_steps, h,
                                                                   stack, wc, defer);
  else
    h = trace_ray<kStats, kAnalytic, kDepth, kDefer, kTlas, kAhs, kInlineMarch>(any_hit, S, o, d, r, tmin, tmax, eps,
                                                                                max_steps, stack, wc, defer);
}

struct Surface {
  float3 n;        // world shading normal facing the ray
  float3 albedo;
  float kr;
  uint32_t chs, is_id;
  uint32_t geom, prim;
};

// Closest-hit inputs of an accepted radiance hit: record (Eq. 1 with r = 0),
// object-space normal, world normal through the inverse transpose.
// grad: the estimator's central-difference gradient at the hit when a march
// job has computed it already (regrouped wavefront), else null. render_pixel
// takes it inline (its two call sites; 1.4 % faster teaser, field and batch
// frames than through the call); the staged wavefront kernels call surface_at.
template <bool kAnalytic = false>
__device__ __forceinline__ Surface surface_body(const SceneView& S, const Hit& h, float3 o, float3 d, float eps,
                                                WorkCounters* wc, const float3* grad) {
  if (wc) ++wc->shaded;
  Surface sf;
  const float4* R = S.inst_rec + 6 * (size_t)h.inst;
  const uint4 info = __ldg(reinterpret_cast<const uint4*>(R + 5));
  const bool tri = (h.leaf & (int)kTriBit) != 0;
  const int leaf = h.leaf & 0x3FFFFFFF;
  uint2 gq = __ldg(S.leaf_gq + leaf);
  uint32_t prim = __ldg(S.leaf_prim + leaf);
  uint32_t rec = 0u + S.sbt_stride_m * gq.x + info.y;
  const uint4 hg = __ldg(S.sbt + rec);   // is, chs, ahs, material
  float4 mat = __ldg(S.materials + hg.w);
  float3 oo, dd;
  to_object(__ldg(R), __ldg(R + 1), __ldg(R + 2), o, d, oo, dd);
  float3 p = madd(oo, h.t, dd);
  float3 no;
  if (tri) {
    const uint32_t* ti = S.indices + 3 * (size_t)prim;
    const float3 v0 = ldf3g(S.vertices + 3 * (size_t)__ldg(ti)), v1 = ldf3g(S.vertices + 3 * (size_t)__ldg(ti + 1)),
                 v2 = ldf3g(S.vertices + 3 * (size_t)__ldg(ti + 2));
    no = cross3(v1 - v0, v2 - v0);
  } else {
    const float4* pp = S.params + 4 * (size_t)prim;
    float4 prm[4] = {__ldg(pp), __ldg(pp + 1), __ldg(pp + 2), __ldg(pp + 3)};
    float hstep = eps * len3(dd);
    no = object_normal<kAnalytic>(hg.x, prm, p, h.attr, hstep, dd, wc, grad);
  }
  // the rows again (L1 hits) rather than held live across the normal's estimates
  const float4 m0 = __ldg(R), m1 = __ldg(R + 1), m2 = __ldg(R + 2);
  float3 nw = f3(fmaf(m0.x, no.x, fmaf(m1.x, no.y, m2.x * no.z)), fmaf(m0.y, no.x, fmaf(m1.y, no.y, m2.y * no.z)),
                 fmaf(m0.z, no.x, fmaf(m1.z, no.y, m2.z * no.z)));
  nw = normalize3(nw);
  if (dot3(nw, d) > 0.f) nw = -nw;
  sf.n = nw;
  sf.albedo = f3(mat.x, mat.y, mat.z);
  sf.kr = mat.w;
  sf.chs = hg.y;
  sf.is_id = hg.x;
  sf.geom = gq.x;
  sf.prim = gq.y;
  return sf;
}

template <bool kAnalytic = false>
__device__ __noinline__ Surface surface_at(const SceneView& S, const Hit& h, float3 o, float3 d, float eps, WorkCounters* wc,
                                           const float3* grad = nullptr) {
  return surface_body<kAnalytic>(S, h, o, d, eps, wc, grad);
}

// Lambert closest-hit shader: ambient + white point light without falloff,
// diffuse gated by visibility: a*k_a + a*I*max(0, n.l)*V, each operation rounded.
__device__ __forceinline__ float light_ndl(const Surface& sf, float3 light, float3 pt) {
  float3 l = normalize3(light - pt);
  return dot3(sf.n, l);
}

__device__ __forceinline__ float3 lambert_rgb(float3 albedo, float ambient, float intensity, float ndl, float vis) {
  float diff = __fmul_rn(__fmul_rn(intensity, fmaxf(0.f, ndl)), vis);
  return f3(__fadd_rn(__fmul_rn(albedo.x, ambient), __fmul_rn(albedo.x, diff)),
            __fadd_rn(__fmul_rn(albedo.y, ambient), __fmul_rn(albedo.y, diff)),
            __fadd_rn(__fmul_rn(albedo.z, ambient), __fmul_rn(albedo.z, diff)));
}

// Mirror blend (1 - k_r) * L + k_r * L_refl.
__device__ __forceinline__ float3 mirror_mix(float3 c, float3 lr, float kr) {
  float w = __fsub_rn(1.f, kr);
  return f3(__fadd_rn(__fmul_rn(c.x, w), __fmul_rn(lr.x, kr)), __fadd_rn(__fmul_rn(c.y, w), __fmul_rn(lr.y, kr)),
            __fadd_rn(__fmul_rn(c.z, w), __fmul_rn(lr.z, kr)));
}

// Scene epsilon from the TLAS root box.
__device__ __forceinline__ float scene_eps(const SceneView& S, float eps_rel) {
  float3 lo = ldf3(S.scene_box), hi = ldf3(S.scene_box + 4);
  return eps_rel * len3(hi - lo);
}

// Ray through the centre of pixel (x, y), row 0 at the top, from the frame's
// orthonormal basis and pixel-to-NDC maps (CameraBasis, computed on the host).
__device__ __forceinline__ float3 camera_ray(const CameraBasis& b, int x, int y) {
  const float ndc_x = fmaf((float)x + 0.5f, b.kx, -1.f) * b.ax;
  const float ndc_y = fmaf((float)y + 0.5f, b.ky, -1.f) * b.ay;
  return normalize3(b.fwd + b.right * ndc_x + b.up * ndc_y);
}

__device__ __forceinline__ float3 miss_rgb(const SceneView& S, uint32_t r, float3 background) {
  return __ldg(S.ray_types + r).x == PR_MISS_BACKGROUND ? background : f3(0.f, 0.f, 0.f);
}

// The per-pixel pipeline of a radiance sample (Section 2.2.3's ray generation
// shader onwards): primary ray, closest-hit shading with its shadow ray, one
// mirror bounce shaded unshadowed, miss shaders. Shared by the single-request
// megakernel and the batched one, so both give the same bits. Writes the AOV
// record when av is given; adds the rays cast to `rays`.
struct PixelParams {
  float3 light, background;
  float light_intensity, ambient;
  uint32_t max_depth, max_steps;
};

// The analytic kernel's per-pixel pipeline with a single traversal site: the
// primary, shadow and mirror rays go through one inlined trace in a loop
// (with an inlined copy per ray kind the kernel's hot code overflowed the
// instruction cache). The same operations in the same order as render_pixel,
// so the same bits.
template <bool kStats, int kDepth, int kTlas, bool kMirror = true>
__device__ __forceinline__ float3 render_pixel_one_site(const SceneView& S, const PixelParams& P, float3 eye, float3 d,
                                                        float eps, TravStack stack, WorkCounters* wc, pr_aov* av,
                                                        uint32_t& rays) {
  enum Stage { kPrimaryRay, kShadowRay, kMirrorRay };
  Stage stage = kPrimaryRay;
  float3 ro = eye, rd = d;
  float rt = INFINITY;
  uint32_t rtype = 0, flags = 0;
  float3 color = f3(0.f, 0.f, 0.f);
  // the primary hit's shading inputs, kept for after the shadow ray
  float3 albedo = color, n = color, pt = color;
  float kr = 0.f, ndl = 0.f, delta = 0.f;
  for (;;) {
    Hit x;
    rays += 1;
    trace_typed<kStats, true, kDepth, false, kTlas>(S, ro, rd, rtype, 0.f, rt, eps, P.max_steps, x, stack, wc);
    float vis = 1.f;
    if (stage == kPrimaryRay) {
      if (x.inst < 0) {
        color = miss_rgb(S, 0, P.background);
        if (av) {
          av->t = -1.f;
          av->inst = av->geom = av->prim = PR_NONE;
          av->n[0] = av->n[1] = av->n[2] = 0.f;
        }
        break;
      }
      flags |= 1u;
      // ro, rd are still the primary ray (eye, d): reading them here leaves
      // eye and d dead after the primary trace unless the mirror needs d
      const Surface sf = surface_body<true>(S, x, ro, rd, eps, wc, nullptr);
      if (av) {
        av->t = x.t;
        av->inst = (uint32_t)x.inst;
        av->geom = sf.geom;
        av->prim = sf.prim;
        av->n[0] = sf.n.x; av->n[1] = sf.n.y; av->n[2] = sf.n.z;
      }
      if (sf.chs != PR_CHS_LAMBERT) break;   // black
      pt = madd(ro, x.t, rd);
      delta = is_sphere_traced(sf.is_id) ? 2.f * eps : eps;
      ndl = light_ndl(sf, P.light, pt);
      albedo = sf.albedo;
      n = sf.n;
      kr = sf.kr;
      if (ndl > 0.f) {
        // shadow ray: offset origin, toward the light, ends at the light
        ro = madd(pt, delta, sf.n);
        const float3 ls = P.light - ro;
        rt = len3(ls);
        rd = ls * (1.f / rt);
        rtype = 1;
        flags |= 2u;
        stage = kShadowRay;
        continue;
      }
    } else if (stage == kShadowRay) {
      vis = x.inst >= 0 ? 0.f : 1.f;
      if (x.inst < 0) flags |= 4u;
    } else {   // the mirror ray's hit, shaded without a shadow ray
      float3 lr;
      if (x.inst >= 0) {
        flags |= 16u;
        const Surface s2 = surface_body<true>(S, x, ro, rd, eps, wc, nullptr);
        if (av) {
          av->refl_t = x.t;
          av->refl_inst = (uint32_t)x.inst;
          av->refl_geom = s2.geom;
          av->refl_prim = s2.prim;
        }
        lr = s2.chs == PR_CHS_LAMBERT
                 ? lambert_rgb(s2.albedo, P.ambient, P.light_intensity, light_ndl(s2, P.light, madd(ro, x.t, rd)), 1.f)
                 : f3(0.f, 0.f, 0.f);
      } else {
        lr = miss_rgb(S, 0, P.background);
      }
      color = mirror_mix(color, lr, kr);
      break;
    }
    color = lambert_rgb(albedo, P.ambient, P.light_intensity, ndl, vis);
    if (kMirror && P.max_depth >= 2 && kr > 0.f) {
      // one mirror bounce from the same offset point
      ro = madd(pt, delta, n);
      rd = normalize3(d - n * (2.f * dot3(d, n)));
      rt = INFINITY;
      rtype = 0;
      flags |= 8u;
      stage = kMirrorRay;
      continue;
    }
    break;
  }
  if (av) {
    if (!(flags & 16u)) {
      av->refl_t = -1.f;
      av->refl_inst = av->refl_geom = av->refl_prim = PR_NONE;
    }
    av->flags = flags;
  }
  return color;
}

// kAhs: the scene (or a batch request's scene) has an any-hit shader on a
// sphere-traced intersection shader. kInlineMarch: the march of the
// sphere-traced shaders is compiled into the traversal instead of called
// (single-request kernel: teaser 13.8 -> 15.5, field 1.94 -> 2.03 Grays/s; the
// one-CTA-per-tile batched kernel: +0.2 %).
// kMirror false: compiled for launches without mirror rays (max_depth 1), so
// none of the mirror bounce's state stays live across the shadow trace.
template <bool kStats, bool kAnalytic = false, int kDepth = kStackDepth, int kTlas = 0, bool kAhs = false,
          bool kInlineMarch = false, bool kMirror = true>
__device__ __forceinline__ float3 render_pixel(const SceneView& S, const PixelParams& P, float3 eye, float3 d, float eps,
                                               TravStack stack, WorkCounters* wc, pr_aov* av, uint32_t& rays) {
  if constexpr (kAnalytic && PR_ANALYTIC_INLINE)
    return render_pixel_one_site<kStats, kDepth, kTlas, kMirror>(S, P, eye, d, eps, stack, wc, av, rays);
  Hit h;
  rays += 1;
  trace_typed<kStats, kAnalytic, kDepth, false, kTlas, kAhs, kInlineMarch>(S, eye, d, 0, 0.f, INFINITY, eps, P.max_steps, h, stack, wc);
  // AOV fields are stored as soon as they are known, so none of them stays
  // live across the shadow and mirror traces
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
    Surface sf = surface_body<kAnalytic>(S, h, eye, d, eps, wc, nullptr);
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
        trace_typed<kStats, kAnalytic, kDepth, false, kTlas, kAhs, kInlineMarch>(S, os, ls * (1.f / dist), 1, 0.f, dist, eps, P.max_steps, sh, stack, wc);
        vis = sh.inst >= 0 ? 0.f : 1.f;
        if (sh.inst < 0) flags |= 4u;
      }
      color = lambert_rgb(sf.albedo, P.ambient, P.light_intensity, ndl, vis);
      if (kMirror && P.max_depth >= 2 && sf.kr > 0.f) {
        // one mirror bounce, its hit shaded without a shadow ray
        float3 orr = madd(pt, delta, sf.n);
        float3 dr = normalize3(d - sf.n * (2.f * dot3(d, sf.n)));
        const float kr = sf.kr;
        Hit rh;
        rays++;
        flags |= 8u;
        trace_typed<kStats, kAnalytic, kDepth, false, kTlas, kAhs, kInlineMarch>(S, orr, dr, 0, 0.f, INFINITY, eps, P.max_steps, rh, stack, wc);
        float3 lr;
        if (rh.inst >= 0) {
          flags |= 16u;
          Surface s2 = surface_body<kAnalytic>(S, rh, orr, dr, eps, wc, nullptr);
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
  if (av) {
    if (!(flags & 16u)) {
      av->refl_t = -1.f;
      av->refl_inst = av->refl_geom = av->refl_prim = PR_NONE;
    }
    av->flags = flags;
  }
  return color;
}


#ifndef PR_SMEM_STACK
#define PR_SMEM_STACK 1
#endif

// Declares `stack` (a TravStack of kDepth entries per thread) for a kernel of
// kThreads threads per CTA.
#if PR_SMEM_STACK
#define PR_DECLARE_STACK_N(kThreads, kDepth)                \
  __shared__ int pr_stack_mem_[(kDepth) * (kThreads)];      \
  const ::pr::TravStack stack{pr_stack_mem_ + threadIdx.x, (kThreads)}
#else
#define PR_DECLARE_STACK_N(kThreads, kDepth)    \
  int pr_stack_mem_[(kDepth)];                   \
  const ::pr::TravStack stack{pr_stack_mem_, 1}
#endif
#define PR_DECLARE_STACK(kThreads) PR_DECLARE_STACK_N(kThreads, ::pr::kStackDepth)

}  // namespace pr
