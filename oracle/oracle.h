/* CPU oracle for the procedural ray tracer — TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow FP64 reference renderer and an FP32 reference LBVH builder.
 * Only tests, the smoke check and the benchmark's CPU-baseline leg may load
 * it. It shares no code, header or constant generator with the CUDA library.
 *
 * Scene arrays follow the entity model of the paper (Section 3.1; Listings
 * 2-10): procedural geometries of AABBs, one BLAS per geometry set, a TLAS
 * of instances, hit groups and shader-table records indexed with Eq. 1.
 */
#ifndef PR_ORACLE_H
#define PR_ORACLE_H
#include <stdint.h>
#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
  uint32_t n_prims, n_geoms, n_blas, n_inst;
  uint32_t n_hit_groups, n_materials, n_records, n_ray_types;
  uint32_t sbt_stride_m;
  const float* aabbs;            /* [n_prims][6] lo.xyz hi.xyz, object space */
  const float* params;           /* [n_prims][16] */
  const uint32_t* geom_prim_begin, *geom_prim_count;   /* [n_geoms] */
  const uint32_t* blas_geom_begin, *blas_geom_count;   /* [n_blas] */
  const float* inst_xform;       /* [n_inst][12] object->world row-major 3x4 */
  const uint32_t* inst_blas, *inst_id, *inst_sbt_offset, *inst_mask;
  const uint32_t* hit_groups;    /* [n_hit_groups][3] is, chs, ahs */
  const float* materials;        /* [n_materials][4] albedo rgb, reflectance */
  const uint32_t* sbt;           /* [n_records][4] hit_group, material, prim_type, instance_index */
  const uint32_t* ray_types;     /* [n_ray_types][2] miss_id, flags */
  const uint32_t* geom_type;     /* [n_geoms] 0 AABBs, 1 triangles; NULL: all AABBs */
  uint32_t n_vertices, n_triangles;
  const float* vertices;         /* [n_vertices][3] */
  const uint32_t* indices;       /* [n_triangles][3]; a triangle geometry's prim range indexes these */
} or_scene;

typedef struct { double eye[3], look_at[3], up[3], vfov_deg; } or_camera;

typedef struct {
  uint32_t width, height, max_depth, max_steps;
  double light_pos[3], light_intensity, eps_rel, ambient, background[3];
} or_params;

/* Per-pixel result. flags: bit0 primary hit, bit1 shadow ray cast, bit2 lit
 * (shadow ray missed), bit3 mirror ray cast, bit4 mirror ray hit, bit5 an
 * Eq. 1 index fell outside the shader table. Ids are -1 on a miss. */
typedef struct {
  double rgb[3];
  double t;
  double n[3];
  double refl_t;
  int32_t inst, geom, prim;
  int32_t refl_inst, refl_geom, refl_prim;
  uint32_t flags;
  uint32_t rays;
} or_pixel;

/* Render the listed pixels (linear index y*width+x; NULL = all pixels). */
int or_render(const or_scene* s, const or_camera* cam, const or_params* p,
              const int64_t* pixels, int64_t n_pixels, or_pixel* out, int n_threads);

/* World bounds of all instances (FP64, 8-corner transform) and the epsilon it implies. */
int or_world_bounds(const or_scene* s, double lo[3], double hi[3]);

/* Single object-space primitive: first surface point at t >= t_lo (analytic;
 * candidates an any-hit shader ahs_id rejects are skipped) or sphere-traced
 * inside [t_lo, t_hi]. Returns 1 on hit and fills t and the object-space
 * normal. eps is the world epsilon; |d| may differ from 1. */
int or_intersect(uint32_t is_id, uint32_t ahs_id, const float* params, const double o[3], const double d[3],
                 double t_lo, double t_hi, double eps, uint32_t max_steps,
                 double* t_out, double n_out[3], uint32_t* steps_out);

/* Distance estimate / signed distance of a sphere-traced primitive at p. */
double or_de(uint32_t is_id, const float* params, const double p[3]);

/* Mandelbulb power map z -> z^n in spherical coordinates (FP64). */
void or_triplex_pow(const double z[3], double n, double out[3]);

/* ---- FP32 reference LBVH (bit-exact target for the device build) -------- */

/* World boxes of all instances in FP32: BLAS root box (union of its AABBs)
 * mapped by object->world with the per-axis min/max form, in a fixed
 * operation order, no fused multiply-add. boxes_out: [n_inst][6]. */
int or_instance_boxes_f32(const or_scene* s, float* boxes_out);

/* LBVH over n boxes: Morton codes of the centroids in the centroid bounds
 * (10 bits per axis), keys (code<<32 | index) sorted, binary radix tree by
 * its top-down definition, child boxes by union.
 *   perm_out   [n]        leaf position -> box index
 *   codes_out  [n]        Morton code of each leaf position
 *   child_out  [n-1][2]   child refs: >= 0 internal node, else (0x80000000 | leaf position)
 *   cbox_out   [n-1][12]  left child lo.xyz hi.xyz, right child lo.xyz hi.xyz
 *   root_box   [6]
 */
int or_lbvh_f32(const float* boxes, uint32_t n, uint32_t* perm_out, uint32_t* codes_out,
                int32_t* child_out, float* cbox_out, float* root_box);

/* PLOC tree over the same boxes and Morton order (Meister & Bittner 2018):
 * mutual nearest neighbours within `radius` positions, by the surface area
 * of their union, merged round by round; nodes numbered n-2 downward in the
 * order they are made (root 0). Same output layout as or_lbvh_f32.
 * Returns 1 for radius 0. */
int or_ploc_f32(const float* boxes, uint32_t n, uint32_t radius, uint32_t* perm_out, uint32_t* codes_out,
                int32_t* child_out, float* cbox_out, float* root_box);

#ifdef __cplusplus
}
#endif
#endif
