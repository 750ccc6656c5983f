// Built-in device "shaders": intersection shaders of the procedural primitive
// types, their normals, and the distance estimators used for sphere tracing.
// All in object space and FP32. The paper names the teaser's shapes (two
// pac-men, a quaternion Julia set, a Mandelbulb; teaser and Figs. 4-6) but
// leaves their shader code to a separate chapter; the shapes below are fixed
// readings of those names plus the SDF primitives of the instanced field.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "pr_device.cuh"

namespace pr {

__device__ __forceinline__ float3 f3(float x, float y, float z) { return make_float3(x, y, z); }
__device__ __forceinline__ float3 operator+(float3 a, float3 b) { return f3(a.x + b.x, a.y + b.y, a.z + b.z); }
__device__ __forceinline__ float3 operator-(float3 a, float3 b) { return f3(a.x - b.x, a.y - b.y, a.z - b.z); }
__device__ __forceinline__ float3 operator-(float3 a) { return f3(-a.x, -a.y, -a.z); }
__device__ __forceinline__ float3 operator*(float3 a, float s) { return f3(a.x * s, a.y * s, a.z * s); }
__device__ __forceinline__ float3 operator*(float s, float3 a) { return f3(a.x * s, a.y * s, a.z * s); }
__device__ __forceinline__ float dot3(float3 a, float3 b) { return fmaf(a.x, b.x, fmaf(a.y, b.y, a.z * b.z)); }
__device__ __forceinline__ float3 cross3(float3 a, float3 b) {
  return f3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
__device__ __forceinline__ float3 normalize3(float3 a) { return a * rsqrtf(dot3(a, a)); }
__device__ __forceinline__ float3 madd(float3 o, float t, float3 d) {   // o + t*d
  return f3(fmaf(t, d.x, o.x), fmaf(t, d.y, o.y), fmaf(t, d.z, o.z));
}
__device__ __forceinline__ float len3(float3 a) { return sqrtf(dot3(a, a)); }
__device__ __forceinline__ float3 ldf3(const float* p) { return f3(p[0], p[1], p[2]); }

// Result attribute of an analytic intersection shader (a DXR attribute struct):
// box: face axis (0..2) + 4 if the face normal is +axis; pac-man: 0 ball, 1/2 wedge plane.
struct IsResult {
  float t;
  uint32_t attr;
  float dist;   // sphere-traced hits: the estimate at t (below eps)
};

// Ray/box slab interval with precomputed 1/d and -o/d: per plane one FMA.
// Three-input minimum / maximum (PTX min.f32 / max.f32 with three sources,
// sm_100 and later): exact, the same value as two nested two-input ones.
__device__ __forceinline__ float fmin3(float a, float b, float c) {
  float r;
  asm("min.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
  return r;
}
__device__ __forceinline__ float fmax3(float a, float b, float c) {
  float r;
  asm("max.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
  return r;
}

// Slab interval clipped to [tmin, tmax] (the parametric range still open).
__device__ __forceinline__ void slab_clip(const float3 lo, const float3 hi, const float3 inv_d, const float3 o_inv,
                                          float tmin, float tmax, float& t0, float& t1) {
  float ax = fmaf(lo.x, inv_d.x, o_inv.x), bx = fmaf(hi.x, inv_d.x, o_inv.x);
  float ay = fmaf(lo.y, inv_d.y, o_inv.y), by = fmaf(hi.y, inv_d.y, o_inv.y);
  float az = fmaf(lo.z, inv_d.z, o_inv.z), bz = fmaf(hi.z, inv_d.z, o_inv.z);
  t0 = fmax3(fminf(ax, bx), fminf(ay, by), fmaxf(fminf(az, bz), tmin));
  t1 = fmin3(fmaxf(ax, bx), fmaxf(ay, by), fminf(fmaxf(az, bz), tmax));
}

__device__ __forceinline__ float3 safe_rcp(float3 d) {
  // slab-test reciprocals (hardware approximation, ~1 ulp), also the box
  // shader's plane distances (within 2 ulp of the IEEE quotient; the oracle's
  // tolerances are 1e-3 of the scene diagonal). A zero component becomes a
  // huge value of its sign, so the axis's slab is (-inf, inf) when the origin
  // lies inside it and empty otherwise.
  const float big = 1e30f;
  return f3(d.x != 0.f ? __fdividef(1.f, d.x) : copysignf(big, d.x),
            d.y != 0.f ? __fdividef(1.f, d.y) : copysignf(big, d.y),
            d.z != 0.f ? __fdividef(1.f, d.z) : copysignf(big, d.z));
}

// ---- any-hit shaders ---------------------------------------------------------
// "Cutout": ignores candidate hits whose object-space point lies in the lower
// half of every band of height 1/4 along y (frac(4y) < 1/2). A hit group's
// any-hit shader runs on each candidate its intersection shader reports, in
// increasing t; an ignored candidate lets the search continue (Section 2.2.3).
__device__ __forceinline__ bool any_hit_accepts(uint32_t ahs, float3 o, float t, float3 d) {
  if (ahs != PR_AHS_CUTOUT) return true;
  float b = 4.f * fmaf(t, d.y, o.y);
  return b - floorf(b) >= 0.5f;
}

// ---- analytic shaders ------------------------------------------------------
// Sphere: closest approach t_c = -(o-c).d/|d|^2, squared half chord from the
// perpendicular distance (numerically kinder than b^2 - ac), first root >= tmin.
// 1/|d|^2 and the half chord's square root by the hardware approximations
// (a few ulp; the 4096-frame analytic run 3 % faster than with IEEE division
// and square root, every oracle comparison within the same bounds).
__device__ __forceinline__ bool is_sphere(const float4 p0, float3 o, float3 d, float tmin, IsResult& r,
                                          uint32_t ahs = PR_NONE) {
  float3 c = f3(p0.x, p0.y, p0.z);
  float R = p0.w;
  float3 f = o - c;
  float a = dot3(d, d);
  float inv_a = __fdividef(1.f, a);
  float tc = -dot3(f, d) * inv_a;
  float3 l = madd(f, tc, d);
  float h2 = (R * R - dot3(l, l)) * inv_a;
  if (h2 < 0.f) return false;
  float h = h2 > 0.f ? h2 * rsqrtf(h2) : 0.f;
  float t = tc - h;
  if (t < tmin || !any_hit_accepts(ahs, o, t, d)) t = tc + h;
  if (t < tmin || !any_hit_accepts(ahs, o, t, d)) return false;
  r.t = t;
  r.attr = 0;
  return true;
}

// Axis-aligned box (centre, half extent): entry point, else exit point when
// the origin is inside; ties on an edge resolve to the lowest axis.
// inv_d: the traversal's slab reciprocals of d (safe_rcp), reused here.
__device__ __forceinline__ bool is_box(const float4 p0, const float4 p1, float3 o, float3 d, float3 inv_d, float tmin,
                                       IsResult& r, uint32_t ahs = PR_NONE) {
  float c[3] = {p0.x, p0.y, p0.z}, e[3] = {p0.w, p1.x, p1.y};
  float oo[3] = {o.x, o.y, o.z}, dd[3] = {d.x, d.y, d.z}, iv[3] = {inv_d.x, inv_d.y, inv_d.z};
  float te = -INFINITY, tx = INFINITY;
  int ea = 0, xa = 0;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    float tn, tf;
    if (dd[k] != 0.f) {
      const float inv = iv[k];
      float t1 = (c[k] - e[k] - oo[k]) * inv, t2 = (c[k] + e[k] - oo[k]) * inv;
      tn = fminf(t1, t2);
      tf = fmaxf(t1, t2);
    } else {
      if (oo[k] < c[k] - e[k] || oo[k] > c[k] + e[k]) return false;
      tn = -INFINITY;
      tf = INFINITY;
    }
    if (tn > te) { te = tn; ea = k; }
    if (tf < tx) { tx = tf; xa = k; }
  }
  if (te > tx) return false;
  if (te >= tmin && any_hit_accepts(ahs, o, te, d)) {
    r.t = te;
    r.attr = (uint32_t)ea | (dd[ea] > 0.f ? 0u : 4u);
  } else if (tx >= tmin && any_hit_accepts(ahs, o, tx, d)) {
    r.t = tx;
    r.attr = (uint32_t)xa | (dd[xa] > 0.f ? 4u : 0u);
  } else {
    return false;
  }
  return true;
}

// Pac-man: ball minus the open wedge {n1.(p-c) < 0, n2.(p-c) < 0} with
// n1 = (-sin a, cos a, 0), n2 = (-sin a, -cos a, 0) (mouth of 2a about +x).
// Ball chord [s0, s1] minus wedge interval (w0, w1); first boundary >= tmin.
__device__ __forceinline__ bool is_pacman(const float4 p0, const float4 p1, float3 o, float3 d, float tmin,
                                          IsResult& r, uint32_t ahs = PR_NONE) {
  float3 c = f3(p0.x, p0.y, p0.z);
  float R = p0.w;
  float sa, ca;
  sincosf(p1.x, &sa, &ca);
  float3 f = o - c;
  float a = dot3(d, d);
  float inv_a = __fdividef(1.f, a);
  float tc = -dot3(f, d) * inv_a;
  float3 l = madd(f, tc, d);
  float h2 = (R * R - dot3(l, l)) * inv_a;
  if (h2 < 0.f) return false;
  float h = h2 > 0.f ? h2 * rsqrtf(h2) : 0.f;
  float s0 = tc - h, s1 = tc + h;
  float w0 = -INFINITY, w1 = INFINITY;
  uint32_t k0 = 0, k1 = 0;
  bool empty = false;
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    float nx = -sa, ny = k == 0 ? ca : -ca;
    float ak = nx * f.x + ny * f.y, bk = nx * d.x + ny * d.y;
    if (bk > 0.f) {
      float tk = -ak / bk;
      if (tk < w1) { w1 = tk; k1 = (uint32_t)k + 1; }
    } else if (bk < 0.f) {
      float tk = -ak / bk;
      if (tk > w0) { w0 = tk; k0 = (uint32_t)k + 1; }
    } else if (ak >= 0.f) {
      empty = true;
    }
  }
  if (w0 >= w1) empty = true;
  // boundary events in increasing t
  float et[4];
  uint32_t ek[4];
  int ne = 0;
  if (empty || w1 <= s0 || w0 >= s1) {
    et[0] = s0; ek[0] = 0; et[1] = s1; ek[1] = 0; ne = 2;
  } else {
    if (w0 > s0) { et[ne] = s0; ek[ne++] = 0; et[ne] = w0; ek[ne++] = k0; }
    if (w1 < s1) { et[ne] = w1; ek[ne++] = k1; et[ne] = s1; ek[ne++] = 0; }
  }
  for (int i = 0; i < ne; ++i) {
    if (et[i] >= tmin && any_hit_accepts(ahs, o, et[i], d)) {
      r.t = et[i];
      r.attr = ek[i];
      return true;
    }
  }
  return false;
}

__device__ __forceinline__ float3 ldf3g(const float* p) { return f3(__ldg(p), __ldg(p + 1), __ldg(p + 2)); }

// Built-in triangle intersection (what DXR does in fixed function), Moller &
// Trumbore 1997: Cramer's rule on o + t d = v0 + u e1 + v e2; u, v >= 0,
// u + v <= 1, t >= tmin, and the any-hit shader's consent.
__device__ __forceinline__ bool is_triangle(float3 v0, float3 v1, float3 v2, float3 o, float3 d, float tmin, float& t,
                                            uint32_t ahs) {
  const float3 e1 = v1 - v0, e2 = v2 - v0;
  const float3 pv = cross3(d, e2);
  const float det = dot3(e1, pv);
  if (det == 0.f) return false;
  const float inv = 1.f / det;
  const float3 tv = o - v0;
  const float u = dot3(tv, pv) * inv;
  if (u < 0.f || u > 1.f) return false;
  const float3 qv = cross3(tv, e1);
  const float v = dot3(d, qv) * inv;
  if (v < 0.f || u + v > 1.f) return false;
  t = dot3(e2, qv) * inv;
  return t >= tmin && any_hit_accepts(ahs, o, t, d);
}

// ---- distance estimators -----------------------------------------------------
// Inside the estimators (the hot loops of sphere tracing) square roots,
// divisions and logarithms use CUDA's fast approximations (rsqrtf,
// __fdividef, __logf; a few ulp): an estimate only steers the march, and its
// hit threshold eps is far coarser than those ulps.
__device__ __forceinline__ float est_sqrt(float x) { return x > 0.f ? x * rsqrtf(x) : 0.f; }
__device__ __forceinline__ float est_div(float a, float b) { return __fdividef(a, b); }
__device__ __forceinline__ float sdf_torus(const float4 p0, float3 p) {
  float qx = est_sqrt(fmaf(p.x, p.x, p.z * p.z)) - p0.x;
  return est_sqrt(fmaf(qx, qx, p.y * p.y)) - p0.y;
}

__device__ __forceinline__ float sdf_roundbox(const float4 p0, float3 p) {
  float rr = p0.w;
  float qx = fabsf(p.x) - (p0.x - rr), qy = fabsf(p.y) - (p0.y - rr), qz = fabsf(p.z) - (p0.z - rr);
  float mx = fmaxf(qx, 0.f), my = fmaxf(qy, 0.f), mz = fmaxf(qz, 0.f);
  float outside = est_sqrt(fmaf(mx, mx, fmaf(my, my, mz * mz)));
  float inside = fminf(fmaxf(qx, fmaxf(qy, qz)), 0.f);
  return outside + inside - rr;
}

__device__ __forceinline__ float sdf_capsule(const float4 p0, float3 p) {
  float y = fminf(fmaxf(p.y, -p0.x), p0.x);
  float dy = p.y - y;
  return est_sqrt(fmaf(p.x, p.x, fmaf(dy, dy, p.z * p.z))) - p0.y;
}

__device__ __forceinline__ float smin_poly(float a, float b, float k) {
  float h = est_div(fmaxf(k - fabsf(a - b), 0.f), k);
  return fminf(a, b) - h * h * k * 0.25f;
}

__device__ __forceinline__ float sdf_metaball4(const float4* prm, float3 p) {
  const float4 p0 = prm[0], p1 = prm[1], p2 = prm[2], p3 = prm[3];
  const float3 q0 = p - f3(p0.x, p0.y, p0.z), q1 = p - f3(p0.w, p1.x, p1.y);
  const float3 q2 = p - f3(p1.z, p1.w, p2.x), q3 = p - f3(p2.y, p2.z, p2.w);
  float d0 = est_sqrt(dot3(q0, q0)) - p3.x;
  float d1 = est_sqrt(dot3(q1, q1)) - p3.y;
  float d2 = est_sqrt(dot3(q2, q2)) - p3.z;
  float d3 = est_sqrt(dot3(q3, q3)) - p3.w;
  const float k = 0.2f;
  return smin_poly(smin_poly(smin_poly(d0, d1, k), d2, k), d3, k);
}

// Quaternion Julia set (q.x real, slice w = 0). Tracks |q'|^2 so that no
// square root is needed per iteration: |q'_{n+1}|^2 = 4 |q_n|^2 |q'_n|^2.
// DE = 0.5 |q| ln|q| / |q'| = 0.25 ln(|q|^2) sqrt(|q|^2 / |q'|^2) once escaped, 0 inside.
// Written as state / step / estimate of one iteration.
struct JuliaState {
  float qx, qy, qz, qw, r2, md2;
};
__device__ __forceinline__ JuliaState julia_start(float3 p) {
  return JuliaState{p.x, p.y, p.z, 0.f, fmaf(p.x, p.x, fmaf(p.y, p.y, p.z * p.z)), 1.f};
}
// q <- q^2 + c; returns true once |q|^2 exceeds the escape radius squared
__device__ __forceinline__ bool julia_step(JuliaState& s, const float4 c, float esc2) {
  s.md2 *= 4.f * s.r2;
  const float nx = fmaf(s.qx, s.qx, -fmaf(s.qy, s.qy, fmaf(s.qz, s.qz, s.qw * s.qw))) + c.x;
  const float tx = 2.f * s.qx;
  const float ny = fmaf(tx, s.qy, c.y), nz = fmaf(tx, s.qz, c.z), nw = fmaf(tx, s.qw, c.w);
  s.qx = nx; s.qy = ny; s.qz = nz; s.qw = nw;
  s.r2 = fmaf(s.qx, s.qx, fmaf(s.qy, s.qy, fmaf(s.qz, s.qz, s.qw * s.qw)));
  return s.r2 > esc2;
}
__device__ __forceinline__ float julia_estimate(const JuliaState& s) {
  return 0.25f * __logf(s.r2) * est_sqrt(est_div(s.r2, s.md2));
}
__device__ __forceinline__ float de_julia(const float4 c, const float4 p1, float3 p, uint32_t* it = nullptr) {
  const int iters = (int)p1.x;
  const float esc2 = p1.y * p1.y;
  JuliaState s = julia_start(p);
  for (int i = 0; i < iters; ++i) {
    if (it) ++*it;
    if (julia_step(s, c, esc2)) return julia_estimate(s);
  }
  return 0.f;
}

// Mandelbulb, power 8, trig-free: with rho = |z.xy|, (z.z + i rho)^8 gives
// r^8 (cos 8theta + i sin 8theta) and ((x + i y)/rho)^8 gives e^{8 i phi};
// z^8 = (Im w8 * Re u8, Im w8 * Im u8, Re w8). dr <- 8 r^7 dr + 1.
// DE = 0.5 ln(r) r / dr once |z| > bailout, 0 inside.
struct BulbState {
  float x, y, z, dr, n2;
};
__device__ __forceinline__ BulbState bulb_start(float3 p) { return BulbState{p.x, p.y, p.z, 1.f, 0.f}; }
// z <- z^8 + c; returns true once |z|^2 exceeds the bailout squared
__device__ __forceinline__ bool bulb_step(BulbState& s, float3 c, float bail2) {
  const float x = s.x, y = s.y, z = s.z;
  const float x2 = x * x, y2 = y * y, z2 = z * z;
  const float rho2 = x2 + y2;
  const float r2 = rho2 + z2;
  const float r = est_sqrt(r2);
  const float r6 = r2 * r2 * r2;
  s.dr = fmaf(8.f * r6 * r, s.dr, 1.f);
  const float rho = est_sqrt(rho2);
  // w = (z + i rho)^2, ^4, ^8
  const float a = z2 - rho2, b = 2.f * z * rho;
  const float a2 = fmaf(a, a, -b * b), b2 = 2.f * a * b;
  const float a3 = fmaf(a2, a2, -b2 * b2), b3 = 2.f * a2 * b2;
  // u^2 = (x + i y)^2 / rho^2, then ^4, ^8
  float ux, uy;
  if (rho2 > 0.f) {
    const float ir = est_div(1.f, rho2);
    ux = (x2 - y2) * ir;
    uy = 2.f * x * y * ir;
  } else {
    ux = 1.f;
    uy = 0.f;
  }
  const float vx = fmaf(ux, ux, -uy * uy), vy = 2.f * ux * uy;
  const float sx = fmaf(vx, vx, -vy * vy), sy = 2.f * vx * vy;
  s.x = fmaf(b3, sx, c.x);
  s.y = fmaf(b3, sy, c.y);
  s.z = a3 + c.z;
  s.n2 = fmaf(s.x, s.x, fmaf(s.y, s.y, s.z * s.z));
  return s.n2 > bail2;
}
__device__ __forceinline__ float bulb_estimate(const BulbState& s) {
  const float rn = est_sqrt(s.n2);
  return est_div(0.5f * __logf(rn) * rn, s.dr);
}
__device__ __forceinline__ float de_mandelbulb(const float4 p0, float3 p, uint32_t* it = nullptr) {
  const int iters = (int)p0.y;
  const float bail2 = p0.z * p0.z;
  BulbState s = bulb_start(p);
  for (int i = 0; i < iters; ++i) {
    if (it) ++*it;
    if (bulb_step(s, p, bail2)) return bulb_estimate(s);
  }
  return 0.f;
}

// Work counters of the instrumented kernel variant (null in the timed kernel).
struct WorkCounters {
  uint32_t tlas_nodes, blas_nodes, instances, leaves, sbt_lookups;
  uint32_t is_calls[PR_IS_COUNT];
  uint32_t de_evals[PR_IS_COUNT];
  uint32_t frac_iters[2];   // Julia, Mandelbulb loop trips
  uint32_t shaded, rays;
  uint32_t tlas_nodes4;     // 4-wide TLAS node visits
  uint32_t tlas_nodes8;     // 8-wide TLAS node visits (float nodes)
  uint32_t tlas_nodes8q;    // 8-wide TLAS node visits (quantised nodes)
};
static_assert(sizeof(WorkCounters) == 4 * PR_WORK_COUNTERS, "counter layout is part of the ABI");

// Central-difference stencil of the estimate at p (six estimates at p +/- h
// along each axis), for the normal of a sphere-traced hit. The closed-form
// SDFs are evaluated side by side (six independent chains overlap); the
// fractal estimates one point after another, each running to its own escape
// (measured: interleaving their iterations runs every point to the slowest
// one's count, which costs more than the overlap gains). Returns
// (d(+x) - d(-x), d(+y) - d(-y), d(+z) - d(-z)).
template <class DE>
__device__ __forceinline__ float3 stencil_one_by_one(float3 p, float h, DE de) {
  float gx = 0.f, gy = 0.f, gz = 0.f;
#pragma unroll 1
  for (int k = 0; k < 6; ++k) {
    const float sh = (k & 1) ? -h : h;
    const int ax = k >> 1;
    const float v = de(f3(ax == 0 ? p.x + sh : p.x, ax == 1 ? p.y + sh : p.y, ax == 2 ? p.z + sh : p.z));
    if (ax == 0) gx = (k & 1) ? gx - v : v;
    else if (ax == 1) gy = (k & 1) ? gy - v : v;
    else gz = (k & 1) ? gz - v : v;
  }
  return f3(gx, gy, gz);
}

// Inline at its call sites (the surface reconstruction of a sphere-traced hit):
// teaser 15.5 -> 15.7 Grays/s, field and batch within 0.7 % faster.
static __device__ __forceinline__ float3 de_stencil(uint32_t id, const float4* prm, float3 p, float h,
                                                 WorkCounters* wc = nullptr) {
  if (wc) wc->de_evals[id < PR_IS_COUNT ? id : 0] += 6;
  const float3 pt[6] = {f3(p.x + h, p.y, p.z), f3(p.x - h, p.y, p.z), f3(p.x, p.y + h, p.z),
                        f3(p.x, p.y - h, p.z), f3(p.x, p.y, p.z + h), f3(p.x, p.y, p.z - h)};
  float v[6];
  const float4 p0 = prm[0];
  switch (id) {
    case PR_IS_JULIA:
    case PR_IS_JULIA_CUT: {
      const float4 p1 = prm[1], b = prm[2];
      const bool cut = id == PR_IS_JULIA_CUT;
      uint32_t* it = wc ? &wc->frac_iters[0] : nullptr;
      return stencil_one_by_one(p, h, [&](float3 q) {
        const float dj = de_julia(p0, p1, q, it);
        // the Julia set cut by the half-space n.p <= d (Fig. 5)
        return cut ? fmaxf(dj, fmaf(p1.z, q.x, fmaf(p1.w, q.y, b.x * q.z)) - b.y) : dj;
      });
    }
    case PR_IS_MANDELBULB: {
      uint32_t* it = wc ? &wc->frac_iters[1] : nullptr;
      return stencil_one_by_one(p, h, [&](float3 q) { return de_mandelbulb(p0, q, it); });
    }
    case PR_IS_TORUS:
#pragma unroll
      for (int k = 0; k < 6; ++k) v[k] = sdf_torus(p0, pt[k]);
      break;
    case PR_IS_ROUNDBOX:
#pragma unroll
      for (int k = 0; k < 6; ++k) v[k] = sdf_roundbox(p0, pt[k]);
      break;
    case PR_IS_CAPSULE:
#pragma unroll
      for (int k = 0; k < 6; ++k) v[k] = sdf_capsule(p0, pt[k]);
      break;
    case PR_IS_METABALL4:
#pragma unroll
      for (int k = 0; k < 6; ++k) v[k] = sdf_metaball4(prm, pt[k]);
      break;
    default:
#pragma unroll
      for (int k = 0; k < 6; ++k) v[k] = INFINITY;
  }
  return f3(v[0] - v[1], v[2] - v[3], v[4] - v[5]);
}

__device__ __forceinline__ bool is_sphere_traced(uint32_t id) { return id >= PR_IS_TORUS && id <= PR_IS_JULIA_CUT; }

// The estimate of a fractal shader (Julia, Mandelbulb, cut Julia) at p, with
// its parameter rows in registers: the arithmetic of the sphere-tracing loop
// and of the normal stencil, for march jobs run outside the traversal.
__device__ __forceinline__ float fractal_de(uint32_t id, const float4 p0, const float4 p1, const float4 p2, float3 p) {
  if (id == PR_IS_MANDELBULB) return de_mandelbulb(p0, p);
  const float dj = de_julia(p0, p1, p);
  if (id == PR_IS_JULIA_CUT) return fmaxf(dj, fmaf(p1.z, p.x, fmaf(p1.w, p.y, p2.x * p.z)) - p2.y);
  return dj;
}

// Sphere tracing (Hart 1996) inside [t_lo, t_hi]: estimates are converted to
// world units with 1/|d|; hit when below eps, give up past t_hi or after
// max_steps estimates. The estimate is inlined into the loop (one branch on
// the shader id per march, parameters kept in registers); the conversion is
// rounded on its own so no multiply-add forms across the estimate's result.
// A hit also returns the estimate there (IsResult::dist): an any-hit shader
// that ignores it restarts the march past it (run_intersection).
template <class DE>
__device__ __forceinline__ IsResult march(DE de, float3 o, float3 d, float inv_len, float t_lo, float t_hi, float eps,
                                          uint32_t max_steps) {
  IsResult r{0.f, 0u, 0.f};
  float t = t_lo;
  for (uint32_t s = 0; s < max_steps; ++s) {
    if (t > t_hi) return r;
    const float dist = __fmul_rn(de(madd(o, t, d)), inv_len);
    if (dist < eps) {
      r.t = t;
      r.attr = s + 1;   // >= 1 marks a hit
      r.dist = dist;
      return r;
    }
    t += dist;
  }
  return r;
}

// The march of a sphere-traced intersection shader; attr of the result is 0
// on a miss.
static __device__ __forceinline__ IsResult sphere_trace_body(uint32_t id, const float4* prm, float3 o, float3 d,
                                                             float inv_len, float t_lo, float t_hi, float eps,
                                                             uint32_t max_steps, WorkCounters* wc) {
  uint32_t* de_ctr = wc ? &wc->de_evals[id < PR_IS_COUNT ? id : 0] : nullptr;
  uint32_t* jit = wc ? &wc->frac_iters[0] : nullptr;
  uint32_t* mit = wc ? &wc->frac_iters[1] : nullptr;
  const float4 p0 = __ldg(prm);
  switch (id) {
    case PR_IS_TORUS:
      return march([&](float3 p) { if (de_ctr) ++*de_ctr; return sdf_torus(p0, p); }, o, d, inv_len, t_lo, t_hi, eps,
                   max_steps);
    case PR_IS_ROUNDBOX:
      return march([&](float3 p) { if (de_ctr) ++*de_ctr; return sdf_roundbox(p0, p); }, o, d, inv_len, t_lo, t_hi, eps,
                   max_steps);
    case PR_IS_CAPSULE:
      return march([&](float3 p) { if (de_ctr) ++*de_ctr; return sdf_capsule(p0, p); }, o, d, inv_len, t_lo, t_hi, eps,
                   max_steps);
    case PR_IS_METABALL4: {
      const float4 q[4] = {p0, __ldg(prm + 1), __ldg(prm + 2), __ldg(prm + 3)};
      return march([&](float3 p) { if (de_ctr) ++*de_ctr; return sdf_metaball4(q, p); }, o, d, inv_len, t_lo, t_hi, eps,
                   max_steps);
    }
    case PR_IS_JULIA: {
      const float4 p1 = __ldg(prm + 1);
      return march([&](float3 p) { if (de_ctr) ++*de_ctr; return de_julia(p0, p1, p, jit); }, o, d, inv_len, t_lo, t_hi,
                   eps, max_steps);
    }
    case PR_IS_MANDELBULB:
      return march([&](float3 p) { if (de_ctr) ++*de_ctr; return de_mandelbulb(p0, p, mit); }, o, d, inv_len, t_lo, t_hi,
                   eps, max_steps);
    case PR_IS_JULIA_CUT: {   // the Julia set cut by the half-space n.p <= d (Fig. 5)
      const float4 a = __ldg(prm + 1), b = __ldg(prm + 2);
      return march(
          [&](float3 p) {
            if (de_ctr) ++*de_ctr;
            const float plane = fmaf(a.z, p.x, fmaf(a.w, p.y, b.x * p.z)) - b.y;
            return fmaxf(de_julia(p0, a, p, jit), plane);
          },
          o, d, inv_len, t_lo, t_hi, eps, max_steps);
    }
    default: return IsResult{0.f, 0u, 0.f};
  }
}

// The same out of line: one copy of the march serves every call site.
static __device__ __noinline__ IsResult sphere_trace(uint32_t id, const float4* prm, float3 o, float3 d, float inv_len,
                                                     float t_lo, float t_hi, float eps, uint32_t max_steps,
                                                     WorkCounters* wc = nullptr) {
  return sphere_trace_body(id, prm, o, d, inv_len, t_lo, t_hi, eps, max_steps, wc);
}

// Object-space normal at the accepted hit (called once per shaded hit).
// kAnalytic: only analytic shaders occur (no estimator stencil compiled in).
template <bool kAnalytic = false>
__device__ __forceinline__ float3 object_normal(uint32_t id, const float4* prm, float3 p, uint32_t attr, float h,
                                                float3 d, WorkCounters* wc = nullptr, const float3* grad = nullptr) {
  switch (id) {
    case PR_IS_SPHERE: {
      float4 p0 = prm[0];
      return (p - f3(p0.x, p0.y, p0.z)) * (1.f / p0.w);
    }
    case PR_IS_BOX: {
      uint32_t ax = attr & 3u;
      float s = (attr & 4u) ? 1.f : -1.f;
      return f3(ax == 0 ? s : 0.f, ax == 1 ? s : 0.f, ax == 2 ? s : 0.f);
    }
    case PR_IS_PACMAN: {
      float4 p0 = prm[0];
      if (attr == 0) return (p - f3(p0.x, p0.y, p0.z)) * (1.f / p0.w);
      float sa, ca;
      sincosf(prm[1].x, &sa, &ca);
      return f3(sa, attr == 1 ? -ca : ca, 0.f);   // -n_k
    }
    default: {
      if (kAnalytic) return -normalize3(d);
      const float3 g = grad ? *grad : de_stencil(id, prm, p, h, wc);
      float gl2 = dot3(g, g);
      return gl2 > 0.f ? g * rsqrtf(gl2) : -normalize3(d);
    }
  }
}

}  // namespace pr
