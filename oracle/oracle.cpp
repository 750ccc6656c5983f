// CPU oracle for the procedural ray tracer — TEST INFRASTRUCTURE ONLY.
//
// Plain, slow and straightforward on purpose: brute force over every
// instance, geometry and AABB primitive, all arithmetic in FP64, no
// acceleration structure, no blocking or reordering. Only tests, the smoke
// check and the benchmark's CPU-baseline leg may load this library; the CUDA
// library shares no code with it.
//
// The paper (Proceduray, da Silva et al.) documents DXR host code. It fixes
// the pipeline stages (Section 2.2.3: ray generation, miss, closest-hit,
// intersection shaders; hit groups), the shader-table indexing rule (Eq. 1),
// one BLAS per geometry with a TLAS of all instances (Section 3.1.5) and the
// record layout of the sample scene (Listing 10). It names but does not print
// the device shaders (pac-man CSG, quaternion Julia set, Mandelbulb; teaser,
// Figs. 4-6): their formulas here are the readings stated beside each function.
//
// Parity: every function below is pinned by tests against closed forms,
// brute force or invariants (ray-sphere and ray-box closed forms, pac-man
// reductions to sphere and plane, dense sign sampling for sphere tracing,
// the no-overshoot invariant of the distance estimators, an independent
// complex-power form of the Mandelbulb map, exhaustive Eq. 1 enumeration,
// the top-down radix-tree definition for the LBVH).
#include "oracle.h"

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <limits>
#include <thread>
#include <vector>

namespace {

// ---- shader ids (scene input format) -------------------------------------
constexpr uint32_t kSphere = 0, kBox = 1, kPacman = 2, kTorus = 3, kRoundbox = 4,
                   kCapsule = 5, kMetaball4 = 6, kJulia = 7, kMandelbulb = 8, kJuliaCut = 9;
constexpr uint32_t kNone = 0xFFFFFFFFu;
constexpr uint32_t kChsLambert = 0;
constexpr uint32_t kAhsCutout = 0;
constexpr uint32_t kGeomTriangles = 1;
constexpr uint32_t kTriangleHit = 1000;   // marks a hit on built-in triangle geometry
constexpr uint32_t kMissBackground = 0, kMissShadow = 1;
constexpr uint32_t kTerminateOnFirstHit = 1;
constexpr double kMetaballK = 0.2;
constexpr double kInf = std::numeric_limits<double>::infinity();

bool is_sphere_traced(uint32_t id) { return id >= kTorus && id <= kJuliaCut; }

// ---- small vector algebra ----------------------------------------------
struct V3 { double x, y, z; };
V3 operator+(V3 a, V3 b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
V3 operator-(V3 a, V3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
V3 operator*(V3 a, double s) { return {a.x * s, a.y * s, a.z * s}; }
V3 operator*(double s, V3 a) { return a * s; }
V3 operator-(V3 a) { return {-a.x, -a.y, -a.z}; }
double dot(V3 a, V3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
V3 cross(V3 a, V3 b) { return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x}; }
double len(V3 a) { return std::sqrt(dot(a, a)); }
V3 normalize(V3 a) { return a * (1.0 / len(a)); }
double comp(V3 a, int k) { return k == 0 ? a.x : (k == 1 ? a.y : a.z); }
V3 axis(int k, double s) { V3 v{0, 0, 0}; if (k == 0) v.x = s; else if (k == 1) v.y = s; else v.z = s; return v; }
V3 from(const double* p) { return {p[0], p[1], p[2]}; }
V3 fromf(const float* p) { return {p[0], p[1], p[2]}; }

// Affine map x -> L x + t stored row-major 3x4.
struct Affine {
  double m[3][4];
  V3 point(V3 p) const {
    return {m[0][0] * p.x + m[0][1] * p.y + m[0][2] * p.z + m[0][3],
            m[1][0] * p.x + m[1][1] * p.y + m[1][2] * p.z + m[1][3],
            m[2][0] * p.x + m[2][1] * p.y + m[2][2] * p.z + m[2][3]};
  }
  V3 vec(V3 v) const {
    return {m[0][0] * v.x + m[0][1] * v.y + m[0][2] * v.z,
            m[1][0] * v.x + m[1][1] * v.y + m[1][2] * v.z,
            m[2][0] * v.x + m[2][1] * v.y + m[2][2] * v.z};
  }
  // L^T v (maps an object-space normal to world space when this is world->object)
  V3 vec_transposed(V3 v) const {
    return {m[0][0] * v.x + m[1][0] * v.y + m[2][0] * v.z,
            m[0][1] * v.x + m[1][1] * v.y + m[2][1] * v.z,
            m[0][2] * v.x + m[1][2] * v.y + m[2][2] * v.z};
  }
};

Affine affine_from(const float* x12) {
  Affine a;
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 4; ++c) a.m[r][c] = x12[r * 4 + c];
  return a;
}

// Inverse of an affine map by the adjugate of its 3x3 part.
Affine affine_inverse(const Affine& a) {
  const double (*m)[4] = a.m;
  double c00 = m[1][1] * m[2][2] - m[1][2] * m[2][1];
  double c01 = m[1][2] * m[2][0] - m[1][0] * m[2][2];
  double c02 = m[1][0] * m[2][1] - m[1][1] * m[2][0];
  double det = m[0][0] * c00 + m[0][1] * c01 + m[0][2] * c02;
  double id = 1.0 / det;
  Affine r;
  r.m[0][0] = c00 * id;
  r.m[0][1] = (m[0][2] * m[2][1] - m[0][1] * m[2][2]) * id;
  r.m[0][2] = (m[0][1] * m[1][2] - m[0][2] * m[1][1]) * id;
  r.m[1][0] = c01 * id;
  r.m[1][1] = (m[0][0] * m[2][2] - m[0][2] * m[2][0]) * id;
  r.m[1][2] = (m[0][2] * m[1][0] - m[0][0] * m[1][2]) * id;
  r.m[2][0] = c02 * id;
  r.m[2][1] = (m[0][1] * m[2][0] - m[0][0] * m[2][1]) * id;
  r.m[2][2] = (m[0][0] * m[1][1] - m[0][1] * m[1][0]) * id;
  for (int i = 0; i < 3; ++i)
    r.m[i][3] = -(r.m[i][0] * m[0][3] + r.m[i][1] * m[1][3] + r.m[i][2] * m[2][3]);
  return r;
}

// ---- ray / box slab interval ----------------------------------------------
// Interval [t_enter, t_exit] of the ray inside the closed box; false if empty.
// A zero direction component keeps the axis unconstrained when the origin lies
// inside the slab and empties the interval otherwise.
bool slab_interval(V3 o, V3 d, V3 lo, V3 hi, double& te, double& tx, int* enter_axis = nullptr,
                   int* exit_axis = nullptr) {
  te = -kInf;
  tx = kInf;
  int ea = 0, xa = 0;
  for (int k = 0; k < 3; ++k) {
    double ok = comp(o, k), dk = comp(d, k), lk = comp(lo, k), hk = comp(hi, k);
    double tn, tf;
    if (dk != 0.0) {
      double t1 = (lk - ok) / dk, t2 = (hk - ok) / dk;
      tn = std::min(t1, t2);
      tf = std::max(t1, t2);
    } else {
      if (ok < lk || ok > hk) return false;
      tn = -kInf;
      tf = kInf;
    }
    if (tn > te) { te = tn; ea = k; }   // ties keep the lowest axis index
    if (tf < tx) { tx = tf; xa = k; }
  }
  if (enter_axis) *enter_axis = ea;
  if (exit_axis) *exit_axis = xa;
  return te <= tx;
}

// ---- analytic intersection shaders (object space) -------------------------
struct IsHit { double t; V3 n; uint32_t steps; };

// Sphere (centre c, radius R): roots of |o + t d - c|^2 = R^2; the first root
// with t >= tmin (the far root when the origin is inside). Normal (p - c) / R.
// Any-hit "cutout" shader: ignores candidate hits whose object-space point
// lies in the lower half of every band of height 1/4 along y (frac(4y) < 1/2).
// A hit group's any-hit shader runs on every candidate an intersection shader
// reports (Section 2.2.3); an ignored candidate lets the search continue.
bool any_hit_accepts(uint32_t ahs, V3 p) {
  if (ahs != kAhsCutout) return true;
  double b = 4.0 * p.y;
  return b - std::floor(b) >= 0.5;
}

bool is_sphere(const float* prm, V3 o, V3 d, double tmin, IsHit& h, uint32_t ahs) {
  V3 c = fromf(prm);
  double R = prm[3];
  V3 oc = o - c;
  double a = dot(d, d), b = dot(oc, d), cc = dot(oc, oc) - R * R;
  double disc = b * b - a * cc;
  if (disc < 0.0) return false;
  double sq = std::sqrt(disc);
  double t0 = (-b - sq) / a, t1 = (-b + sq) / a;
  double t;
  if (t0 >= tmin && any_hit_accepts(ahs, o + t0 * d)) t = t0;
  else if (t1 >= tmin && any_hit_accepts(ahs, o + t1 * d)) t = t1;
  else return false;
  h.t = t;
  h.n = (o + t * d - c) * (1.0 / R);
  h.steps = 0;
  return true;
}

// Axis-aligned box (centre c, half extent e): the slab entry point when it is
// at or beyond tmin (normal: entering face, against d), else the exit point.
bool is_box(const float* prm, V3 o, V3 d, double tmin, IsHit& h, uint32_t ahs) {
  V3 c = fromf(prm), e = fromf(prm + 3);
  double te, tx;
  int ea, xa;
  if (!slab_interval(o, d, c - e, c + e, te, tx, &ea, &xa)) return false;
  if (te >= tmin && any_hit_accepts(ahs, o + te * d)) {
    h.t = te;
    h.n = axis(ea, comp(d, ea) > 0 ? -1.0 : 1.0);
  } else if (tx >= tmin && any_hit_accepts(ahs, o + tx * d)) {
    h.t = tx;
    h.n = axis(xa, comp(d, xa) > 0 ? 1.0 : -1.0);
  } else {
    return false;
  }
  h.steps = 0;
  return true;
}

// Pac-man: the ball |p - c| <= R minus the open wedge W = {n1.(p-c) < 0 and
// n2.(p-c) < 0}, n1 = (-sin a, cos a, 0), n2 = (-sin a, -cos a, 0): a mouth of
// opening 2a about +x, running along z. Along the ray the ball is one interval
// [s0, s1] and the wedge one interval (w0, w1); the solid is their difference.
// The hit is its first boundary point with t >= tmin. Normals: the ball's
// (p - c) / R, or -n_k on the face of wedge plane k.
bool is_pacman(const float* prm, V3 o, V3 d, double tmin, IsHit& h, uint32_t ahs) {
  V3 c = fromf(prm);
  double R = prm[3], a = prm[4];
  V3 oc = o - c;
  double qa = dot(d, d), qb = dot(oc, d), qc = dot(oc, oc) - R * R;
  double disc = qb * qb - qa * qc;
  if (disc < 0.0) return false;
  double sq = std::sqrt(disc);
  double s0 = (-qb - sq) / qa, s1 = (-qb + sq) / qa;

  V3 nrm[2] = {{-std::sin(a), std::cos(a), 0.0}, {-std::sin(a), -std::cos(a), 0.0}};
  double w0 = -kInf, w1 = kInf;
  int p0 = -1, p1 = -1;
  bool wedge_empty = false;
  for (int k = 0; k < 2; ++k) {
    double ak = dot(nrm[k], oc), bk = dot(nrm[k], d);
    if (bk > 0.0) {
      double tk = -ak / bk;
      if (tk < w1) { w1 = tk; p1 = k; }
    } else if (bk < 0.0) {
      double tk = -ak / bk;
      if (tk > w0) { w0 = tk; p0 = k; }
    } else if (ak >= 0.0) {
      wedge_empty = true;
    }
  }
  if (w0 >= w1) wedge_empty = true;

  struct Ev { double t; int kind; };   // kind: -1 ball, else wedge plane index
  Ev ev[4];
  int ne = 0;
  if (wedge_empty || w1 <= s0 || w0 >= s1) {
    ev[ne++] = {s0, -1};
    ev[ne++] = {s1, -1};
  } else {
    if (w0 > s0) { ev[ne++] = {s0, -1}; ev[ne++] = {w0, p0}; }
    if (w1 < s1) { ev[ne++] = {w1, p1}; ev[ne++] = {s1, -1}; }
  }
  for (int i = 0; i < ne; ++i) {
    if (ev[i].t >= tmin && any_hit_accepts(ahs, o + ev[i].t * d)) {
      h.t = ev[i].t;
      h.n = ev[i].kind < 0 ? (o + h.t * d - c) * (1.0 / R) : -nrm[ev[i].kind];
      h.steps = 0;
      return true;
    }
  }
  return false;
}

// Built-in triangle intersection (DXR's fixed-function test), written as
// Moller & Trumbore 1997: t and barycentrics (u, v) from Cramer's rule on
// o + t d = v0 + u e1 + v e2; a hit needs u, v >= 0, u + v <= 1 and t >= tmin
// (and the any-hit shader's consent). Normal: e1 x e2, normalised.
bool is_triangle(V3 v0, V3 v1, V3 v2, V3 o, V3 d, double tmin, IsHit& h, uint32_t ahs) {
  V3 e1 = v1 - v0, e2 = v2 - v0;
  V3 pv = cross(d, e2);
  double det = dot(e1, pv);
  if (det == 0.0) return false;
  double inv = 1.0 / det;
  V3 tv = o - v0;
  double u = dot(tv, pv) * inv;
  if (u < 0.0 || u > 1.0) return false;
  V3 qv = cross(tv, e1);
  double v = dot(d, qv) * inv;
  if (v < 0.0 || u + v > 1.0) return false;
  double t = dot(e2, qv) * inv;
  if (t < tmin || !any_hit_accepts(ahs, o + t * d)) return false;
  h.t = t;
  h.n = normalize(cross(e1, e2));
  h.steps = 0;
  return true;
}

// ---- distance estimators (object space) -----------------------------------
// Exact Euclidean signed distances of the torus (ring radius R about y, tube
// radius r), the rounded box (outer half extent b, rounding radius rr) and the
// capsule (segment y in [-h, h], radius r), written from their geometry.
double sdf_torus(const float* prm, V3 p) {
  double R = prm[0], r = prm[1];
  double qx = std::sqrt(p.x * p.x + p.z * p.z) - R;
  return std::sqrt(qx * qx + p.y * p.y) - r;
}

double sdf_roundbox(const float* prm, V3 p) {
  double rr = prm[3];
  double q[3] = {std::fabs(p.x) - (prm[0] - rr), std::fabs(p.y) - (prm[1] - rr), std::fabs(p.z) - (prm[2] - rr)};
  double outside = std::sqrt(std::max(q[0], 0.0) * std::max(q[0], 0.0) + std::max(q[1], 0.0) * std::max(q[1], 0.0) +
                             std::max(q[2], 0.0) * std::max(q[2], 0.0));
  double inside = std::min(std::max(q[0], std::max(q[1], q[2])), 0.0);
  return outside + inside - rr;
}

double sdf_capsule(const float* prm, V3 p) {
  double hh = prm[0], r = prm[1];
  double y = std::min(std::max(p.y, -hh), hh);
  return len(p - V3{0.0, y, 0.0}) - r;
}

// Metaball cluster: four balls (centres prm[0..11], radii prm[12..15]) merged
// with the polynomial smooth minimum smin(a,b) = min(a,b) - k/4 * h^2,
// h = max(k - |a-b|, 0) / k, k = 0.2. Its gradient is a convex combination of
// the balls' unit gradients, so it stays 1-Lipschitz and safe to sphere trace.
double smin_poly(double a, double b, double k) {
  double hh = std::max(k - std::fabs(a - b), 0.0) / k;
  return std::min(a, b) - hh * hh * k * 0.25;
}

double sdf_metaball4(const float* prm, V3 p) {
  double dist[4];
  for (int i = 0; i < 4; ++i) dist[i] = len(p - fromf(prm + 3 * i)) - prm[12 + i];
  double m = smin_poly(dist[0], dist[1], kMetaballK);
  m = smin_poly(m, dist[2], kMetaballK);
  return smin_poly(m, dist[3], kMetaballK);
}

// Quaternion Julia set (Hart, Sandin & Kauffman 1989), 3-D slice q = (x,y,z,0)
// with q.x the real part. Iterate q <- q^2 + c and |q'| <- 2 |q| |q'| (|q'_0| = 1)
// for at most prm[4] iterations, stopping once |q| exceeds the escape radius
// prm[5]. Escaped: DE = 0.5 |q| ln|q| / |q'|; not escaped: inside, DE = 0.
double de_julia(const float* prm, V3 p) {
  double c[4] = {prm[0], prm[1], prm[2], prm[3]};
  int iters = (int)prm[4];
  double esc2 = (double)prm[5] * (double)prm[5];
  double q[4] = {p.x, p.y, p.z, 0.0};
  double md = 1.0;
  for (int i = 0; i < iters; ++i) {
    double qn = std::sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
    md = 2.0 * qn * md;
    double n0 = q[0] * q[0] - q[1] * q[1] - q[2] * q[2] - q[3] * q[3] + c[0];
    double n1 = 2.0 * q[0] * q[1] + c[1];
    double n2 = 2.0 * q[0] * q[2] + c[2];
    double n3 = 2.0 * q[0] * q[3] + c[3];
    q[0] = n0; q[1] = n1; q[2] = n2; q[3] = n3;
    double r2 = q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3];
    if (r2 > esc2) {
      double r = std::sqrt(r2);
      return 0.5 * r * std::log(r) / md;
    }
  }
  return 0.0;
}

// Mandelbulb power map in spherical coordinates (White & Nylander 2009):
// r = |z|, theta = acos(z_z / r), phi = atan2(z_y, z_x);
// z^n = r^n (sin n.theta cos n.phi, sin n.theta sin n.phi, cos n.theta).
V3 triplex_pow(V3 z, double n) {
  double r = len(z);
  if (r == 0.0) return {0.0, 0.0, 0.0};
  double th = std::acos(std::max(-1.0, std::min(1.0, z.z / r))) * n;
  double ph = std::atan2(z.y, z.x) * n;
  double rn = std::pow(r, n);
  return {rn * std::sin(th) * std::cos(ph), rn * std::sin(th) * std::sin(ph), rn * std::cos(th)};
}

// Mandelbulb (power prm[0], at most prm[1] iterations, bailout prm[2]):
// dr <- n r^(n-1) dr + 1 (dr_0 = 1), z <- z^n + p, stop once |z| > bailout.
// Escaped: DE = 0.5 ln(r) r / dr; not escaped: inside, DE = 0.
double de_mandelbulb(const float* prm, V3 p) {
  double n = prm[0];
  int iters = (int)prm[1];
  double bail = prm[2];
  V3 z = p;
  double dr = 1.0;
  for (int i = 0; i < iters; ++i) {
    double r = len(z);
    dr = n * std::pow(r, n - 1.0) * dr + 1.0;
    z = triplex_pow(z, n) + p;
    double rz = len(z);
    if (rz > bail) return 0.5 * std::log(rz) * rz / dr;
  }
  return 0.0;
}

// Julia set cut by a plane (the paper's Fig. 5): the set intersected with the
// half-space n.p <= d (unit n = prm[6..8], d = prm[9]). The larger of the two
// distance bounds bounds the distance to the intersection from below.
double de_julia_cut(const float* prm, V3 p) {
  V3 n = fromf(prm + 6);
  return std::max(de_julia(prm, p), dot(n, p) - (double)prm[9]);
}

double distance_estimate(uint32_t id, const float* prm, V3 p) {
  switch (id) {
    case kTorus: return sdf_torus(prm, p);
    case kRoundbox: return sdf_roundbox(prm, p);
    case kCapsule: return sdf_capsule(prm, p);
    case kMetaball4: return sdf_metaball4(prm, p);
    case kJulia: return de_julia(prm, p);
    case kMandelbulb: return de_mandelbulb(prm, p);
    case kJuliaCut: return de_julia_cut(prm, p);
    default: return kInf;
  }
}

// Sphere tracing (Hart 1996) inside [t_lo, t_hi]: at each step the object-space
// estimate is converted to world units by 1/|d| (d is the object-space image of
// a unit world direction); a hit is declared when it drops below eps, else t
// advances by it; the march gives up past t_hi or after max_steps estimates.
// Normal: normalised central-difference gradient with step h = eps |d|
// (eps expressed in object units); a zero gradient falls back to -d.
// Every march point whose estimate is below eps is a candidate, reported in
// increasing t to the hit group's any-hit shader (Section 2.2.3); an ignored
// candidate lets the march go on by the estimate's magnitude, at least eps
// (through the solid, where an exact SDF is negative, and out of it), so the
// next candidate is the next point in or on the surface that the march visits.
bool is_sphere_trace(uint32_t id, const float* prm, V3 o, V3 d, double t_lo, double t_hi, double eps,
                     uint32_t max_steps, IsHit& h, uint32_t ahs = kNone) {
  double dl = len(d);
  double inv_len = 1.0 / dl;
  double t = t_lo;
  for (uint32_t s = 0; s < max_steps; ++s) {
    if (t > t_hi) return false;
    V3 p = o + t * d;
    double dist = distance_estimate(id, prm, p) * inv_len;
    if (dist < eps && !any_hit_accepts(ahs, p)) {
      t += std::max(std::fabs(dist), eps);
      continue;
    }
    if (dist < eps) {
      double hh = eps * dl;
      V3 g{distance_estimate(id, prm, p + V3{hh, 0, 0}) - distance_estimate(id, prm, p - V3{hh, 0, 0}),
           distance_estimate(id, prm, p + V3{0, hh, 0}) - distance_estimate(id, prm, p - V3{0, hh, 0}),
           distance_estimate(id, prm, p + V3{0, 0, hh}) - distance_estimate(id, prm, p - V3{0, 0, hh})};
      double gl = len(g);
      h.t = t;
      h.n = gl > 0.0 ? g * (1.0 / gl) : -d * inv_len;
      h.steps = s + 1;
      return true;
    }
    t += dist;
  }
  return false;
}

// Intersection-shader dispatch by shader id. Analytic shaders report their
// first surface point at t >= tmin; sphere-traced ones march [t_lo, t_hi].
bool intersect(uint32_t id, const float* prm, V3 o, V3 d, double tmin, double t_lo, double t_hi, double eps,
               uint32_t max_steps, IsHit& h, uint32_t ahs = kNone) {
  switch (id) {
    case kSphere: return is_sphere(prm, o, d, tmin, h, ahs);
    case kBox: return is_box(prm, o, d, tmin, h, ahs);
    case kPacman: return is_pacman(prm, o, d, tmin, h, ahs);
    default:
      if (is_sphere_traced(id)) return is_sphere_trace(id, prm, o, d, t_lo, t_hi, eps, max_steps, h, ahs);
      return false;
  }
}

// ---- scene preparation ---------------------------------------------------
struct Prepared {
  const or_scene* s;
  std::vector<Affine> w2o;          // world -> object per instance
  std::vector<V3> wlo, whi;         // world box per instance (culling only)
  std::vector<V3> blo, bhi;         // object-space root box per BLAS
  V3 scene_lo, scene_hi;
  double eps;
};

bool is_triangle_geom(const or_scene* s, uint32_t geom) {
  return s->geom_type && s->geom_type[geom] == kGeomTriangles;
}

// Object-space box of one primitive: an AABB as given, or a triangle's vertex bounds.
void prim_box(const or_scene* s, uint32_t geom, uint32_t prim, float out[6]) {
  if (!is_triangle_geom(s, geom)) {
    std::memcpy(out, s->aabbs + 6 * (size_t)prim, 6 * sizeof(float));
    return;
  }
  const uint32_t* t = s->indices + 3 * (size_t)prim;
  for (int k = 0; k < 3; ++k) {
    out[k] = INFINITY;
    out[3 + k] = -INFINITY;
  }
  for (int c = 0; c < 3; ++c)
    for (int k = 0; k < 3; ++k) {
      float v = s->vertices[3 * (size_t)t[c] + k];
      out[k] = std::min(out[k], v);
      out[3 + k] = std::max(out[3 + k], v);
    }
}

void blas_root_box(const or_scene* s, uint32_t b, V3& lo, V3& hi) {
  lo = {kInf, kInf, kInf};
  hi = {-kInf, -kInf, -kInf};
  for (uint32_t g = 0; g < s->blas_geom_count[b]; ++g) {
    uint32_t geom = s->blas_geom_begin[b] + g;
    for (uint32_t q = 0; q < s->geom_prim_count[geom]; ++q) {
      float bx[6];
      prim_box(s, geom, s->geom_prim_begin[geom] + q, bx);
      lo = {std::min(lo.x, (double)bx[0]), std::min(lo.y, (double)bx[1]), std::min(lo.z, (double)bx[2])};
      hi = {std::max(hi.x, (double)bx[3]), std::max(hi.y, (double)bx[4]), std::max(hi.z, (double)bx[5])};
    }
  }
}

void prepare(const or_scene* s, Prepared& P, double eps_rel) {
  P.s = s;
  P.blo.resize(s->n_blas);
  P.bhi.resize(s->n_blas);
  for (uint32_t b = 0; b < s->n_blas; ++b) blas_root_box(s, b, P.blo[b], P.bhi[b]);
  P.w2o.resize(s->n_inst);
  P.wlo.resize(s->n_inst);
  P.whi.resize(s->n_inst);
  P.scene_lo = {kInf, kInf, kInf};
  P.scene_hi = {-kInf, -kInf, -kInf};
  for (uint32_t k = 0; k < s->n_inst; ++k) {
    Affine o2w = affine_from(s->inst_xform + 12 * (size_t)k);
    P.w2o[k] = affine_inverse(o2w);
    V3 lo = P.blo[s->inst_blas[k]], hi = P.bhi[s->inst_blas[k]];
    V3 wl{kInf, kInf, kInf}, wh{-kInf, -kInf, -kInf};
    for (int corner = 0; corner < 8; ++corner) {
      V3 p{(corner & 1) ? hi.x : lo.x, (corner & 2) ? hi.y : lo.y, (corner & 4) ? hi.z : lo.z};
      V3 w = o2w.point(p);
      wl = {std::min(wl.x, w.x), std::min(wl.y, w.y), std::min(wl.z, w.z)};
      wh = {std::max(wh.x, w.x), std::max(wh.y, w.y), std::max(wh.z, w.z)};
    }
    // pad by a relative hair so that FP64 rounding never culls a grazing ray
    V3 pad = (wh - wl) * 1e-9 + V3{1e-12, 1e-12, 1e-12};
    P.wlo[k] = wl - pad;
    P.whi[k] = wh + pad;
    P.scene_lo = {std::min(P.scene_lo.x, wl.x), std::min(P.scene_lo.y, wl.y), std::min(P.scene_lo.z, wl.z)};
    P.scene_hi = {std::max(P.scene_hi.x, wh.x), std::max(P.scene_hi.y, wh.y), std::max(P.scene_hi.z, wh.z)};
  }
  P.eps = s->n_inst ? eps_rel * len(P.scene_hi - P.scene_lo) : eps_rel;
}

// ---- traversal: brute force closest / any hit ---------------------------
struct Hit {
  bool valid = false;
  double t = kInf;
  int32_t inst = -1, geom = -1, prim = -1;
  uint32_t record = 0, is_id = kNone;
  V3 n_world{0, 0, 0};
};

bool key_less(int32_t i0, int32_t g0, int32_t p0, int32_t i1, int32_t g1, int32_t p1) {
  if (i0 != i1) return i0 < i1;
  if (g0 != g1) return g0 < g1;
  return p0 < p1;
}

// One TraceRay (Section 2.2.3): every instance whose mask passes, every AABB
// of its BLAS that the ray enters within [tmin, t_closest], the shader-table
// record a = r + m*g + i (Eq. 1, h_s = 0 and h_p = one record), and the
// intersection shader of that record's hit group. A report is accepted when
// tmin <= t < t_closest; an exact tie keeps the lower (instance, geometry,
// primitive) key. With terminate-on-first-hit the first accepted report ends
// the search. sbt_error is set when an Eq. 1 index falls outside the table.
Hit trace_ray(const Prepared& P, V3 o, V3 d, uint32_t r, double tmin, double tmax, uint32_t max_steps,
              bool& sbt_error) {
  const or_scene* s = P.s;
  bool first_hit = (s->ray_types[2 * r + 1] & kTerminateOnFirstHit) != 0;
  Hit best;
  best.t = tmax;
  for (uint32_t k = 0; k < s->n_inst; ++k) {
    if ((s->inst_mask[k] & 0xFFu) == 0) continue;
    double te, tx;
    if (!slab_interval(o, d, P.wlo[k], P.whi[k], te, tx)) continue;
    if (std::max(te, tmin) > std::min(tx, best.t)) continue;
    const Affine& w2o = P.w2o[k];
    V3 oo = w2o.point(o), dd = w2o.vec(d);
    uint32_t b = s->inst_blas[k];
    for (uint32_t g = 0; g < s->blas_geom_count[b]; ++g) {
      uint32_t geom = s->blas_geom_begin[b] + g;
      const bool tri = is_triangle_geom(s, geom);
      for (uint32_t q = 0; q < s->geom_prim_count[geom]; ++q) {
        uint32_t prim = s->geom_prim_begin[geom] + q;
        IsHit ih;
        uint64_t rec = (uint64_t)r + (uint64_t)s->sbt_stride_m * g + s->inst_sbt_offset[k];
        uint32_t is_id;
        if (tri) {
          // built-in triangle test; the record still supplies the hit group
          const uint32_t* t = s->indices + 3 * (size_t)prim;
          V3 v0 = fromf(s->vertices + 3 * (size_t)t[0]), v1 = fromf(s->vertices + 3 * (size_t)t[1]),
             v2 = fromf(s->vertices + 3 * (size_t)t[2]);
          if (rec >= s->n_records) { sbt_error = true; continue; }
          uint32_t hg = s->sbt[4 * rec + 0];
          if (hg >= s->n_hit_groups) { sbt_error = true; continue; }
          if (!is_triangle(v0, v1, v2, oo, dd, tmin, ih, s->hit_groups[3 * hg + 2])) continue;
          is_id = kTriangleHit;
        } else {
          const float* bx = s->aabbs + 6 * (size_t)prim;
          double be, bxit;
          if (!slab_interval(oo, dd, fromf(bx), fromf(bx + 3), be, bxit)) continue;
          double t_lo = std::max(be, tmin), t_hi = std::min(bxit, best.t);
          if (t_lo > t_hi) continue;
          if (rec >= s->n_records) { sbt_error = true; continue; }
          uint32_t hg = s->sbt[4 * rec + 0];
          if (hg >= s->n_hit_groups) { sbt_error = true; continue; }
          is_id = s->hit_groups[3 * hg + 0];
          uint32_t ahs_id = s->hit_groups[3 * hg + 2];
          if (!intersect(is_id, s->params + 16 * (size_t)prim, oo, dd, tmin, t_lo, t_hi, P.eps, max_steps, ih, ahs_id))
            continue;
        }
        if (ih.t < tmin) continue;
        bool accept = ih.t < best.t ||
                      (best.valid && ih.t == best.t && key_less((int32_t)k, (int32_t)g, (int32_t)q, best.inst, best.geom, best.prim));
        if (!accept) continue;
        best.valid = true;
        best.t = ih.t;
        best.inst = (int32_t)k;
        best.geom = (int32_t)g;
        best.prim = (int32_t)q;
        best.record = (uint32_t)rec;
        best.is_id = is_id;
        V3 nw = normalize(w2o.vec_transposed(ih.n));
        best.n_world = dot(nw, d) > 0.0 ? -nw : nw;
        if (first_hit) return best;
      }
    }
  }
  return best;
}

V3 background(const or_params* p) { return from(p->background); }

// Closest-hit "Lambert" shader: ambient + diffuse from a white point light
// without falloff, diffuse gated by the shadow-ray visibility.
V3 lambert(const or_params* p, const float* mat, V3 n, V3 pt, double vis, double* ndl_out) {
  V3 l = normalize(from(p->light_pos) - pt);
  double ndl = dot(n, l);
  if (ndl_out) *ndl_out = ndl;
  V3 alb = fromf(mat);
  return alb * p->ambient + alb * (p->light_intensity * std::max(0.0, ndl) * vis);
}

void render_pixel(const Prepared& P, const or_camera* cam, const or_params* p, int64_t pix, or_pixel& out) {
  const or_scene* s = P.s;
  std::memset(&out, 0, sizeof(out));
  out.inst = out.geom = out.prim = -1;
  out.refl_inst = out.refl_geom = out.refl_prim = -1;
  out.t = -1.0;
  out.refl_t = -1.0;
  int64_t x = pix % p->width, y = pix / p->width;

  // Ray generation: pinhole through the pixel centre, image row 0 at the top.
  V3 eye = from(cam->eye);
  V3 f = normalize(from(cam->look_at) - eye);
  V3 rt = normalize(cross(from(cam->up), f));
  V3 up = cross(f, rt);
  double th = std::tan(cam->vfov_deg * M_PI / 360.0);
  double aspect = (double)p->width / (double)p->height;
  double ndc_x = (((double)x + 0.5) / p->width * 2.0 - 1.0) * th * aspect;
  double ndc_y = -(((double)y + 0.5) / p->height * 2.0 - 1.0) * th;
  V3 d = normalize(f + ndc_x * rt + ndc_y * up);

  bool sbt_err = false;
  uint32_t rays = 1;
  Hit h = trace_ray(P, eye, d, 0, 0.0, kInf, p->max_steps, sbt_err);
  V3 color;
  uint32_t flags = 0;
  if (!h.valid) {
    color = s->ray_types[0] == kMissBackground ? background(p) : V3{0, 0, 0};
  } else {
    flags |= 1u;
    out.t = h.t;
    out.inst = h.inst;
    out.geom = h.geom;
    out.prim = h.prim;
    out.n[0] = h.n_world.x;
    out.n[1] = h.n_world.y;
    out.n[2] = h.n_world.z;
    uint32_t hg = s->sbt[4 * h.record + 0];
    uint32_t chs = s->hit_groups[3 * hg + 1];
    const float* mat = s->materials + 4 * (size_t)s->sbt[4 * h.record + 1];
    if (chs != kChsLambert) {
      color = {0, 0, 0};
    } else {
      V3 pt = eye + h.t * d;
      V3 n = h.n_world;
      double delta = is_sphere_traced(h.is_id) ? 2.0 * P.eps : P.eps;
      double ndl;
      lambert(p, mat, n, pt, 1.0, &ndl);
      double vis = 1.0;
      if (ndl > 0.0) {
        // Shadow ray: offset origin, toward the light, ends at the light.
        V3 os = pt + n * delta;
        V3 ls = from(p->light_pos) - os;
        double dist = len(ls);
        rays++;
        flags |= 2u;
        Hit sh = trace_ray(P, os, ls * (1.0 / dist), 1, 0.0, dist, p->max_steps, sbt_err);
        vis = sh.valid ? 0.0 : 1.0;
        if (!sh.valid) flags |= 4u;
      }
      color = lambert(p, mat, n, pt, vis, nullptr);
      double kr = mat[3];
      if (p->max_depth >= 2 && kr > 0.0) {
        // One mirror bounce; its hit is shaded without a shadow ray.
        V3 orr = pt + n * delta;
        V3 dr = normalize(d - n * (2.0 * dot(d, n)));
        rays++;
        flags |= 8u;
        Hit rh = trace_ray(P, orr, dr, 0, 0.0, kInf, p->max_steps, sbt_err);
        V3 lr;
        if (rh.valid) {
          flags |= 16u;
          out.refl_t = rh.t;
          out.refl_inst = rh.inst;
          out.refl_geom = rh.geom;
          out.refl_prim = rh.prim;
          uint32_t hg2 = s->sbt[4 * rh.record + 0];
          const float* mat2 = s->materials + 4 * (size_t)s->sbt[4 * rh.record + 1];
          lr = s->hit_groups[3 * hg2 + 1] == kChsLambert ? lambert(p, mat2, rh.n_world, orr + rh.t * dr, 1.0, nullptr)
                                                          : V3{0, 0, 0};
        } else {
          lr = s->ray_types[0] == kMissBackground ? background(p) : V3{0, 0, 0};
        }
        color = color * (1.0 - kr) + lr * kr;
      }
    }
  }
  if (sbt_err) flags |= 32u;
  out.rgb[0] = color.x;
  out.rgb[1] = color.y;
  out.rgb[2] = color.z;
  out.flags = flags;
  out.rays = rays;
}

// ---- FP32 LBVH reference ------------------------------------------------
// Spread the 10 low bits of v to every third bit (bit b -> bit 3b).
uint32_t spread_bits(uint32_t v) {
  uint32_t r = 0;
  for (int b = 0; b < 10; ++b)
    if ((v >> b) & 1u) r |= 1u << (3 * b);
  return r;
}

int clz64(uint64_t v) {
  int n = 0;
  for (int b = 63; b >= 0; --b) {
    if ((v >> b) & 1u) break;
    ++n;
  }
  return n;
}

struct TreeBuild {
  const std::vector<uint64_t>& keys;
  const float* boxes;
  const std::vector<uint32_t>& perm;
  int32_t* child;
  float* cbox;
};

void box_union(const float* a, const float* b, float* out) {
  for (int k = 0; k < 3; ++k) {
    out[k] = std::min(a[k], b[k]);
    out[3 + k] = std::max(a[3 + k], b[3 + k]);
  }
}

// Binary radix tree by definition: a range [first, last] of sorted distinct
// keys splits after the last key that shares more leading bits with keys[first]
// than keys[last] does. The left child covers [first, s] and is numbered s,
// the right child covers [s+1, last] and is numbered s+1 (the root is 0); a
// one-key range is a leaf. Returns the node's box in out_box.
void build_range(TreeBuild& T, uint32_t first, uint32_t last, uint32_t node, float* out_box) {
  int common = clz64(T.keys[first] ^ T.keys[last]);
  uint32_t s = first;
  for (uint32_t i = first; i < last; ++i)
    if (clz64(T.keys[first] ^ T.keys[i]) > common) s = i;
  float lbox[6], rbox[6];
  int32_t lref, rref;
  if (s == first) {
    lref = (int32_t)(0x80000000u | s);
    std::memcpy(lbox, T.boxes + 6 * (size_t)T.perm[s], sizeof(lbox));
  } else {
    lref = (int32_t)s;
    build_range(T, first, s, s, lbox);
  }
  if (s + 1 == last) {
    rref = (int32_t)(0x80000000u | (s + 1));
    std::memcpy(rbox, T.boxes + 6 * (size_t)T.perm[s + 1], sizeof(rbox));
  } else {
    rref = (int32_t)(s + 1);
    build_range(T, s + 1, last, s + 1, rbox);
  }
  T.child[2 * (size_t)node + 0] = lref;
  T.child[2 * (size_t)node + 1] = rref;
  std::memcpy(T.cbox + 12 * (size_t)node, lbox, sizeof(lbox));
  std::memcpy(T.cbox + 12 * (size_t)node + 6, rbox, sizeof(rbox));
  box_union(lbox, rbox, out_box);
}

// Morton keys of the LBVH: code << 32 | leaf index, unsorted.
std::vector<uint64_t> morton_keys(const float* boxes, uint32_t n) {
  // Centroids (lo + hi) * 0.5 and their bounds.
  std::vector<float> cen(3 * (size_t)n);
  float clo[3] = {INFINITY, INFINITY, INFINITY}, chi[3] = {-INFINITY, -INFINITY, -INFINITY};
  for (uint32_t i = 0; i < n; ++i)
    for (int k = 0; k < 3; ++k) {
      float c = (boxes[6 * (size_t)i + k] + boxes[6 * (size_t)i + 3 + k]) * 0.5f;
      cen[3 * (size_t)i + k] = c;
      clo[k] = std::min(clo[k], c);
      chi[k] = std::max(chi[k], c);
    }
  // Morton code: per axis u = (c - lo) / extent (0 when the extent is 0),
  // q = floor(u * 1024) clamped to 1023, bits interleaved x, y, z (x highest).
  std::vector<uint64_t> keys(n);
  for (uint32_t i = 0; i < n; ++i) {
    uint32_t q[3];
    for (int k = 0; k < 3; ++k) {
      float ext = chi[k] - clo[k];
      float u = ext > 0.0f ? (cen[3 * (size_t)i + k] - clo[k]) / ext : 0.0f;
      float qf = u * 1024.0f;
      uint32_t qi = (uint32_t)qf;
      q[k] = qi > 1023u ? 1023u : qi;
    }
    uint32_t code = (spread_bits(q[0]) << 2) | (spread_bits(q[1]) << 1) | spread_bits(q[2]);
    keys[i] = ((uint64_t)code << 32) | i;
  }
  return keys;
}

// Half the surface area of the union of two boxes, dx dy + dy dz + dz dx in
// float, evaluated as fma(dx, dy, fma(dy, dz, dz * dx)) (the precision and
// order the device builder decides merges in); NaN orders last.
float union_half_area(const float* a, const float* b) {
  const float dx = std::max(a[3], b[3]) - std::min(a[0], b[0]);
  const float dy = std::max(a[4], b[4]) - std::min(a[1], b[1]);
  const float dz = std::max(a[5], b[5]) - std::min(a[2], b[2]);
  const float s = std::fma(dx, dy, std::fma(dy, dz, dz * dx));
  return std::isnan(s) ? INFINITY : s;
}

}  // namespace

extern "C" {

int or_render(const or_scene* s, const or_camera* cam, const or_params* p, const int64_t* pixels, int64_t n_pixels,
              or_pixel* out, int n_threads) {
  if (!s || !cam || !p || !out || p->width == 0 || p->height == 0) return 1;
  Prepared P;
  prepare(s, P, p->eps_rel);
  int64_t total = pixels ? n_pixels : (int64_t)p->width * p->height;
  if (n_threads <= 0) n_threads = (int)std::max(1u, std::thread::hardware_concurrency());
  std::atomic<int64_t> next{0};
  const int64_t chunk = 16;
  auto work = [&]() {
    for (;;) {
      int64_t b = next.fetch_add(chunk);
      if (b >= total) break;
      int64_t e = std::min(total, b + chunk);
      for (int64_t i = b; i < e; ++i) render_pixel(P, cam, p, pixels ? pixels[i] : i, out[i]);
    }
  };
  std::vector<std::thread> th;
  for (int t = 1; t < n_threads; ++t) th.emplace_back(work);
  work();
  for (auto& t : th) t.join();
  return 0;
}

int or_world_bounds(const or_scene* s, double lo[3], double hi[3]) {
  Prepared P;
  prepare(s, P, 1.0);
  lo[0] = P.scene_lo.x; lo[1] = P.scene_lo.y; lo[2] = P.scene_lo.z;
  hi[0] = P.scene_hi.x; hi[1] = P.scene_hi.y; hi[2] = P.scene_hi.z;
  return 0;
}

int or_intersect(uint32_t is_id, uint32_t ahs_id, const float* params, const double o[3], const double d[3],
                 double t_lo, double t_hi, double eps, uint32_t max_steps, double* t_out, double n_out[3],
                 uint32_t* steps_out) {
  IsHit h;
  if (!intersect(is_id, params, from(o), from(d), t_lo, t_lo, t_hi, eps, max_steps, h, ahs_id)) return 0;
  *t_out = h.t;
  n_out[0] = h.n.x; n_out[1] = h.n.y; n_out[2] = h.n.z;
  if (steps_out) *steps_out = h.steps;
  return 1;
}

double or_de(uint32_t is_id, const float* params, const double p[3]) { return distance_estimate(is_id, params, from(p)); }

void or_triplex_pow(const double z[3], double n, double out[3]) {
  V3 r = triplex_pow(from(z), n);
  out[0] = r.x; out[1] = r.y; out[2] = r.z;
}

int or_instance_boxes_f32(const or_scene* s, float* boxes_out) {
  std::vector<float> root(6 * (size_t)s->n_blas);
  for (uint32_t b = 0; b < s->n_blas; ++b) {
    float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (uint32_t g = 0; g < s->blas_geom_count[b]; ++g) {
      uint32_t geom = s->blas_geom_begin[b] + g;
      for (uint32_t q = 0; q < s->geom_prim_count[geom]; ++q) {
        float bx[6];
        prim_box(s, geom, s->geom_prim_begin[geom] + q, bx);
        for (int k = 0; k < 3; ++k) {
          lo[k] = std::min(lo[k], bx[k]);
          hi[k] = std::max(hi[k], bx[3 + k]);
        }
      }
    }
    for (int k = 0; k < 3; ++k) { root[6 * b + k] = lo[k]; root[6 * b + 3 + k] = hi[k]; }
  }
  // Per output axis i: t_i + sum_j min/max(m_ij lo_j, m_ij hi_j), accumulated
  // j = 0, 1, 2 in that order, every product and sum rounded to float.
  for (uint32_t k = 0; k < s->n_inst; ++k) {
    const float* m = s->inst_xform + 12 * (size_t)k;
    const float* rb = root.data() + 6 * (size_t)s->inst_blas[k];
    for (int i = 0; i < 3; ++i) {
      float lo = m[4 * i + 3], hi = m[4 * i + 3];
      for (int j = 0; j < 3; ++j) {
        float a = m[4 * i + j] * rb[j];
        float b = m[4 * i + j] * rb[3 + j];
        lo = lo + std::min(a, b);
        hi = hi + std::max(a, b);
      }
      boxes_out[6 * (size_t)k + i] = lo;
      boxes_out[6 * (size_t)k + 3 + i] = hi;
    }
  }
  return 0;
}

int or_lbvh_f32(const float* boxes, uint32_t n, uint32_t* perm_out, uint32_t* codes_out, int32_t* child_out,
                float* cbox_out, float* root_box) {
  if (n == 0) return 0;
  std::vector<uint64_t> keys = morton_keys(boxes, n);
  std::sort(keys.begin(), keys.end());
  std::vector<uint32_t> perm(n);
  for (uint32_t i = 0; i < n; ++i) {
    perm[i] = (uint32_t)(keys[i] & 0xFFFFFFFFu);
    perm_out[i] = perm[i];
    codes_out[i] = (uint32_t)(keys[i] >> 32);
  }
  if (n == 1) {
    std::memcpy(root_box, boxes + 6 * (size_t)perm[0], 6 * sizeof(float));
    return 0;
  }
  TreeBuild T{keys, boxes, perm, child_out, cbox_out};
  build_range(T, 0, n - 1, 0, root_box);
  return 0;
}

// PLOC (parallel locally-ordered clustering, Meister & Bittner 2018), one
// round after another on one thread. The clusters start as the leaves in the
// LBVH's Morton order. In each round every cluster i picks as its nearest
// neighbour the cluster j != i within `radius` positions of it whose pair
// {i, j} is least in the order: surface area of the union, then |i - j|, then
// min(i, j) even before odd, then min(i, j) (a total order on pairs, so the
// least pair of a round is mutual; on equal boxes it pairs 0-1, 2-3, ...
// and halves the list each round); every pair
// of mutual nearest neighbours i < j becomes a new node (left child i, right
// child j) that takes i's place while j leaves the list, the other clusters
// keeping their order. The nodes are numbered n-2, n-3, ... in the order they
// are made (round by round, within a round by position), so the last one is
// the root 0. Same output layout as or_lbvh_f32 (leaves 0x80000000 | sorted
// position).
int or_ploc_f32(const float* boxes, uint32_t n, uint32_t radius, uint32_t* perm_out, uint32_t* codes_out,
                int32_t* child_out, float* cbox_out, float* root_box) {
  if (n == 0) return 0;
  if (radius == 0) return 1;
  std::vector<uint64_t> keys = morton_keys(boxes, n);
  std::sort(keys.begin(), keys.end());
  struct Cluster {
    int32_t ref;
    float box[6];
  };
  std::vector<Cluster> C(n);
  for (uint32_t i = 0; i < n; ++i) {
    const uint32_t leaf = (uint32_t)(keys[i] & 0xFFFFFFFFu);
    perm_out[i] = leaf;
    codes_out[i] = (uint32_t)(keys[i] >> 32);
    C[i].ref = (int32_t)(0x80000000u | i);
    std::memcpy(C[i].box, boxes + 6 * (size_t)leaf, sizeof(C[i].box));
  }
  int64_t next = (int64_t)n - 2;
  while (C.size() > 1) {
    const int64_t m = (int64_t)C.size();
    std::vector<int64_t> nn(m);
    for (int64_t i = 0; i < m; ++i) {
      int64_t best_j = -1;
      float best = INFINITY;
      for (int64_t j = std::max<int64_t>(0, i - radius); j <= std::min<int64_t>(m - 1, i + radius); ++j) {
        if (j == i) continue;
        const float a = union_half_area(C[i].box, C[j].box);
        bool take = best_j < 0 || a < best;
        if (!take && a == best) {
          const int64_t d = std::llabs(i - j), db = std::llabs(i - best_j);
          const int64_t lo = std::min(i, j), lob = std::min(i, best_j);
          take = d != db ? d < db : (lo & 1) != (lob & 1) ? (lo & 1) == 0 : lo < lob;
        }
        if (take) {
          best = a;
          best_j = j;
        }
      }
      nn[i] = best_j;
    }
    std::vector<Cluster> D;
    for (int64_t i = 0; i < m; ++i) {
      const int64_t j = nn[i];
      const bool mutual = nn[j] == i;
      if (mutual && j < i) continue;   // merged into the node made at j
      if (!mutual) {
        D.push_back(C[i]);
        continue;
      }
      if (next < 0) return 2;          // more merges than internal nodes: cannot happen
      const int64_t node = next--;
      child_out[2 * node + 0] = C[i].ref;
      child_out[2 * node + 1] = C[j].ref;
      std::memcpy(cbox_out + 12 * node, C[i].box, sizeof(C[i].box));
      std::memcpy(cbox_out + 12 * node + 6, C[j].box, sizeof(C[j].box));
      Cluster u;
      u.ref = (int32_t)node;
      box_union(C[i].box, C[j].box, u.box);
      D.push_back(u);
    }
    C.swap(D);
  }
  std::memcpy(root_box, C[0].box, sizeof(C[0].box));
  return 0;
}

}  // extern "C"
