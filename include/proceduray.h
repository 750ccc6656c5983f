/* proceduray.h — C ABI of the B300 procedural-primitive ray tracer.
 *
 * A software re-design, for one sm_103a GPU, of the pipeline the paper
 * (Proceduray, da Silva, Novello, Lopes, Velho) sets up through DXR:
 * procedural geometry as AABBs with custom intersection shaders (Section
 * 2.2.3), one BLAS per geometry set and a TLAS of all instances (Section
 * 3.1.5), hit groups {intersection, any-hit, closest-hit} and shader-table
 * records reached with the indexing rule of Eq. 1,
 *     a = h_s + h_p * (r + m*g + i),
 * and entries built from <ray, hit group, root arguments> tuples (Section
 * 3.1.7, Listing 10). Traversal that DXR leaves to fixed-function hardware is
 * done in software CUDA; the acceleration structure is an LBVH built on the
 * device from Morton codes and a radix sort.
 *
 * Conventions for every entry point:
 *  - Plain C types only. `stream` is a cudaStream_t passed as void*; NULL is
 *    the legacy default stream. All device work of a call is enqueued on it.
 *  - Host arrays in descriptors are read during the call and may be freed
 *    when it returns. Device output buffers are owned by the caller.
 *  - Synchronous validation errors return a pr_status (nothing is enqueued).
 *    Errors found by kernels (an Eq. 1 index outside the table, a traversal
 *    stack overflow) are OR-ed into the scene's device error word, read with
 *    pr_scene_error. No call throws or aborts.
 *  - pr_last_error() gives a thread-local message for the last failure.
 */
#ifndef PROCEDURAY_H
#define PROCEDURAY_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PR_ABI_VERSION 1u

typedef enum {
  PR_OK = 0,
  PR_ERR_INVALID_ARG = 1,
  PR_ERR_OUT_OF_MEMORY = 2,
  PR_ERR_CUDA = 3,
  PR_ERR_SBT_INDEX = 4,       /* error-word bit 1<<4: Eq. 1 index outside the table */
  PR_ERR_STACK_OVERFLOW = 5,  /* error-word bit 1<<5: traversal stack exhausted */
  PR_ERR_TIMEOUT = 6,
  PR_ERR_NOT_BUILT = 7,       /* pr_trace before pr_build_bvh */
  PR_ERR_BUDGET = 8
} pr_status;

#define PR_NONE 0xFFFFFFFFu

/* Built-in shader ids named by hit groups and ray types, like the exports a
 * DXR hit group names (Listing 3). Intersection shaders: */
#define PR_IS_SPHERE 0u      /* params: centre xyz, radius */
#define PR_IS_BOX 1u         /* params: centre xyz, half extent xyz (also the ground slab) */
#define PR_IS_PACMAN 2u      /* params: centre xyz, radius, mouth half-angle (rad) */
#define PR_IS_TORUS 3u       /* params: ring radius, tube radius (axis y) */
#define PR_IS_ROUNDBOX 4u    /* params: outer half extent xyz, rounding radius */
#define PR_IS_CAPSULE 5u     /* params: half length (axis y), radius */
#define PR_IS_METABALL4 6u   /* params: 4 centres xyz, 4 radii; smooth-min k = 0.2 */
#define PR_IS_JULIA 7u       /* params: c (4), iterations, escape radius */
#define PR_IS_MANDELBULB 8u  /* params: power (8), iterations, bailout */
#define PR_IS_JULIA_CUT 9u   /* params: as Julia, then unit plane normal (3), offset d:
                                the set cut by the half-space n.p <= d (Fig. 5) */
#define PR_IS_COUNT 10u
/* Closest-hit shaders */
#define PR_CHS_LAMBERT 0u
/* Any-hit shaders (run on every candidate hit; may ignore it). PR_AHS_CUTOUT
 * ignores candidates whose object-space point has frac(4*y) < 1/2 (bands cut
 * out of the surface). Every intersection shader reports its candidates in
 * increasing t: the sphere its two roots, the box its entry and exit, the
 * pac-man its boundary events; a sphere-traced shader every march point whose
 * estimate is below eps, the march going on after an ignored one by the
 * estimate's magnitude (at least eps), through the solid and out of it. */
#define PR_AHS_CUTOUT 0u
/* Miss shaders */
#define PR_MISS_BACKGROUND 0u
#define PR_MISS_SHADOW 1u
/* Ray-type flags (what DXR passes as TraceRay flags) */
#define PR_RAY_TERMINATE_ON_FIRST_HIT 1u
#define PR_RAY_SKIP_CLOSEST_HIT 2u   /* accepted as DXR's flag; closest-hit shaders run for radiance rays only */
/* Trace flags */
#define PR_TRACE_WRITE_AOV 1u
#define PR_TRACE_TLAS_BVH2 2u   /* traverse the binary TLAS instead of its 4-wide collapse */
#define PR_TRACE_OUTPUT_RGB 4u  /* the image holds 3 floats per pixel (r, g, b; 12 bytes) instead of
                                   4 (r, g, b, alpha = 1); the values are the same */
/* Geometry kinds */
#define PR_GEOM_AABBS 0u
#define PR_GEOM_TRIANGLES 1u
/* Primitive parameter floats per AABB primitive */
#define PR_PARAMS_PER_PRIM 16u
/* Largest traversal stack; deeper trees set PR_ERR_STACK_OVERFLOW */
#define PR_STACK_DEPTH 64u

typedef struct pr_scene pr_scene;

/* Scene description (host arrays, little-endian), the entity model of the
 * paper's Section 3.1 flattened into arrays:
 *  aabbs            [n_prims][6] float  object-space lo.xyz, hi.xyz (lo <= hi)
 *  params           [n_prims][16] float shape parameters of each AABB primitive
 *  geom_prim_begin/count [n_geoms]      primitives of geometry g (AABBs, or triangles)
 *  blas_geom_begin/count [n_blas]       geometries of each BLAS; the geometry
 *                                       index g of Eq. 1 is the position in it
 *  inst_xform       [n_inst][12] float  object->world, row-major 3x4, invertible
 *  inst_blas, inst_id, inst_sbt_offset, inst_mask [n_inst]
 *                   inst_sbt_offset is Eq. 1's i in records (DXR's
 *                   InstanceContributionToHitGroupIndex); mask 0 hides it
 *  hit_groups       [n_hit_groups][3] uint32 is_id, chs_id, ahs_id (PR_NONE = absent;
 *                   ahs PR_AHS_CUTOUT needs an intersection shader)
 *  materials        [n_materials][4] float albedo rgb, mirror reflectance
 *  sbt              [n_records][4] uint32 hit_group, material, prim_type, instance_index
 *                   (the root arguments of Listing 10)
 *  ray_types        [n_ray_types][2] uint32 miss_id, flags; type 0 is the radiance
 *                   ray (Eq. 1 r = 0), type 1 the shadow ray (r = 1)
 *  sbt_stride_m     Eq. 1 geometry multiplier m */
typedef struct {
  uint32_t struct_size; /* sizeof(pr_scene_desc) */
  uint32_t n_prims, n_geoms, n_blas, n_inst;
  uint32_t n_hit_groups, n_materials, n_records, n_ray_types;
  uint32_t sbt_stride_m;
  const float* aabbs;
  const float* params;
  const uint32_t* geom_prim_begin;
  const uint32_t* geom_prim_count;
  const uint32_t* blas_geom_begin;
  const uint32_t* blas_geom_count;
  const float* inst_xform;
  const uint32_t* inst_blas;
  const uint32_t* inst_id;
  const uint32_t* inst_sbt_offset;
  const uint32_t* inst_mask;
  const uint32_t* hit_groups;
  const float* materials;
  const uint32_t* sbt;
  const uint32_t* ray_types;
  /* Triangle geometry (the built-in triangle intersection of DXR). geom_type
   * [n_geoms] is PR_GEOM_AABBS or PR_GEOM_TRIANGLES (NULL: all AABBs); for a
   * triangle geometry, geom_prim_begin/count index triangles, not AABBs. A
   * BLAS holds one kind only (as in DXR). */
  const uint32_t* geom_type;
  uint32_t n_vertices, n_triangles;
  const float* vertices;     /* [n_vertices][3] object space */
  const uint32_t* indices;   /* [n_triangles][3] vertex indices */
} pr_scene_desc;

/* Pinhole camera (ray generation shader, Section 2.2.3): rays leave eye through
 * pixel centres; vertical field of view in degrees; image row 0 at the top. */
typedef struct {
  float eye[3], look_at[3], up[3], vfov_deg;
} pr_camera;

/* Frame parameters. eps = eps_rel * (diagonal of the TLAS root box) is the
 * sphere-tracing hit threshold in world units; shadow/mirror origins are offset
 * by eps (analytic) or 2*eps (sphere-traced) along the normal. max_depth 1:
 * primary + shadow rays; 2: plus one mirror bounce shaded without shadow. */
typedef struct {
  uint32_t struct_size; /* sizeof(pr_trace_params) */
  uint32_t width, height, max_depth, max_steps, flags;
  float light_pos[3];
  float light_intensity, eps_rel, ambient;
  float background[3];
} pr_trace_params;

/* Optional per-pixel validation output (48 bytes). Ids are 0xFFFFFFFF on a
 * miss; inst is the instance's index in the scene (creation order), geom the
 * geometry index g inside its BLAS, prim the primitive index in the geometry.
 * flags: 1 hit, 2 shadow ray cast, 4 lit, 8 mirror ray cast, 16 mirror hit.
 * n is the world shading normal (facing the ray). Eq. 1 indices outside the
 * table are reported through the scene's error word. */
typedef struct {
  float t;
  uint32_t inst, geom, prim;
  float n[3];
  uint32_t flags;
  float refl_t;
  uint32_t refl_inst, refl_geom, refl_prim;
} pr_aov;

/* ABI version (PR_ABI_VERSION). */
uint32_t pr_version(void);

/* Thread-local message of the last failing call ("" if none). */
const char* pr_last_error(void);

/* Host-only validation of a description (no GPU needed). */
pr_status pr_scene_validate(const pr_scene_desc* desc);

/* Eq. 1 on the host: *out = r + m*g + i with h_s = 0 and h_p = one record.
 * Returns PR_ERR_SBT_INDEX when the index is >= n_records (no write). */
pr_status pr_sbt_index(uint32_t r, uint32_t m, uint32_t g, uint32_t i, uint32_t n_records, uint32_t* out);

/* Validate, allocate one device arena sized for the scene and its BVH build
 * (and a pinned host buffer of the size of its inputs), and copy the
 * description to the device on `stream`. The caller's arrays are read during
 * the call only. The BVH is not built. */
pr_status pr_scene_create(const pr_scene_desc* desc, void* stream, pr_scene** out);

/* Re-upload a description with the same counts into an existing scene
 * (no allocation); marks the BVH stale. The inputs are packed into the
 * scene's pinned buffer during the call and sent with one asynchronous copy on
 * `stream` (the call first waits for the previous upload's copy to finish). */
pr_status pr_scene_upload(pr_scene* scene, const pr_scene_desc* desc, void* stream);

/* Build the two-level BVH on the device (asynchronous on `stream`): each BLAS
 * over its AABBs, the instance world boxes, then the TLAS over the instances.
 * Each level is an LBVH: Morton codes of box centroids in the centroid bounds,
 * keys sorted by a device radix sort, a binary radix tree (Karras 2012) and
 * bottom-up box unions. */
pr_status pr_build_bvh(pr_scene* scene, void* stream);

/* pr_build_bvh of n scenes, the builds of different scenes running
 * concurrently: they are spread over a pool of internal streams (created on
 * the first call per device) that start after the work already enqueued on
 * `stream`, and `stream`'s later work waits for all of them. Asynchronous;
 * the first failing build's status is returned (the others are still
 * enqueued). A scene may appear once (PR_ERR_INVALID_ARG, nothing enqueued,
 * if one appears twice). Calls from several host threads take turns. The launches of a
 * call are kept as a CUDA graph (one per device) and replayed by the next call
 * that builds the same scenes, in the same order, with the same flags: a
 * scene's launches are fixed by its counts, which pr_scene_upload cannot
 * change, so a replay rebuilds every BVH from the scenes' current inputs.
 * Calls with PR_BUILD_TLAS_PLOC or PR_BUILD_TLAS_BVH8_F32, or on a stream that
 * is being captured, launch directly. */
pr_status pr_build_bvh_many(pr_scene* const* scenes, uint32_t n, void* stream);

/* Build options (pr_build_bvh_ex, pr_build_bvh_many_ex). */
#define PR_BUILD_TLAS_PLOC 1u   /* a TLAS of more than 1024 instances is built by
                                   PLOC (parallel locally-ordered clustering,
                                   Meister & Bittner 2018) instead of the LBVH:
                                   the same Morton order, then mutual nearest
                                   neighbours (by the surface area of their
                                   union, within 16 clusters on either side)
                                   merged bottom-up; a tree of lower SAH cost
                                   in the same node layout, built in one
                                   cooperative launch. Smaller TLASes and every
                                   BLAS keep the LBVH. */

#define PR_BUILD_TLAS_PARITY4 2u  /* the 4-wide TLAS (64 or more instances) takes
                                    the binary nodes at even depth as 4-wide
                                    nodes over their grandchildren (by default
                                    each 4-wide node opens its internal child
                                    of largest surface area until it has 4
                                    children: 3 % faster traversal on the
                                    100 000-instance field) */
#define PR_BUILD_TLAS_BVH8 4u     /* an 8-wide TLAS (64 or more instances),
                                    collapsed greedily like the default 4-wide one,
                                    in quantised 96-byte nodes (child bounds as
                                    bytes on a per-node power-of-two grid,
                                    Ylitie et al. 2017), traversed by pr_trace
                                    and pr_trace_frames; batched launches keep
                                    the binary TLAS for such scenes */
#define PR_BUILD_TLAS_BVH8_F32 8u /* as PR_BUILD_TLAS_BVH8 with float nodes
                                    (224 bytes); the first such build of a scene
                                    allocates their buffer (device, 224 B per
                                    instance, freed with the scene) */

/* pr_build_bvh with options (a bitwise or of PR_BUILD_* flags; 0 is
 * pr_build_bvh; at most one of PARITY4, BVH8, BVH8_F32). PR_ERR_INVALID_ARG
 * for an unknown flag or two wide formats; PR_ERR_CUDA when the
 * device refuses the cooperative launch. The clustering launch waits at
 * grid-wide barriers with a 2 s limit; should one run out (its blocks not
 * all resident, which the cooperative launch rules out), the LBVH passes
 * enqueued after it build the TLAS instead and the scene's error word gets
 * bit 1<<PR_ERR_TIMEOUT. Build PLOC scenes of one device from one stream at
 * a time or through pr_build_bvh_many_ex: two clustering launches must not
 * run side by side. */
pr_status pr_build_bvh_ex(pr_scene* scene, uint32_t flags, void* stream);

/* pr_build_bvh_many with options; the clustering launches of the builds run
 * one after another (each waits for the previous one), the rest of the
 * builds concurrently. */
pr_status pr_build_bvh_many_ex(pr_scene* const* scenes, uint32_t n, uint32_t flags, void* stream);

/* Render one frame into out_rgba (device, caller-owned, height*width float4,
 * row-major, alpha = 1; height*width*3 floats with PR_TRACE_OUTPUT_RGB). out_aov (device, height*width pr_aov) is written when
 * params->flags has PR_TRACE_WRITE_AOV, else may be NULL. ray_counter (device
 * uint64, optional) is incremented by the number of rays cast. Asynchronous. */
pr_status pr_trace(pr_scene* scene, const pr_camera* camera, const pr_trace_params* params, float* out_rgba,
                   pr_aov* out_aov, uint64_t* ray_counter, void* stream);

/* Render n_frames frames of the same scene, one camera each (host array), in
 * one launch: frame f goes to out_rgba + f*height*width*4 (and out_aov +
 * f*height*width). */
pr_status pr_trace_frames(pr_scene* scene, const pr_camera* cameras, uint32_t n_frames,
                          const pr_trace_params* params, float* out_rgba, pr_aov* out_aov, uint64_t* ray_counter,
                          void* stream);

/* Work counters of pr_trace_work (uint64 each, in this order): TLAS node
 * visits, BLAS node visits, instance transitions, leaf tests (AABB slab
 * or triangle; the leaf of a one-AABB BLAS is tested by its root box and
 * not counted here), Eq. 1 record lookups, intersection-shader calls per shader id [PR_IS_COUNT],
 * distance-estimate evaluations per shader id [PR_IS_COUNT], Julia
 * iterations, Mandelbulb iterations, shaded hits, rays traced, 4-wide TLAS
 * node visits, 8-wide TLAS node visits (float nodes), 8-wide TLAS node
 * visits (quantised nodes). */
#define PR_WORK_COUNTERS 32u

/* pr_trace_frames with an instrumented kernel variant that also adds the
 * work it did to work_counters (device, PR_WORK_COUNTERS uint64,
 * caller-zeroed). Same images; slower; meant for roofline accounting. */
pr_status pr_trace_work(pr_scene* scene, const pr_camera* cameras, uint32_t n_frames, const pr_trace_params* params,
                        float* out_rgba, uint64_t* work_counters, void* stream);

/* Read and clear the scene's device error word on `stream` (synchronises the
 * stream). Bits: 1<<PR_ERR_SBT_INDEX, 1<<PR_ERR_STACK_OVERFLOW, and
 * 1<<PR_ERR_TIMEOUT when a PLOC build fell back to the LBVH. */
pr_status pr_scene_error(pr_scene* scene, void* stream, uint32_t* error_word);

/* Scene diagonal and TLAS root box as built (synchronises the stream). */
pr_status pr_scene_bounds(pr_scene* scene, void* stream, float box[6]);

/* Copy one built BVH level to host memory (synchronises the stream).
 * level = PR_NONE: the TLAS (leaves are instance indices); else the BLAS with
 * that index (leaves are primitive positions inside the BLAS, geometry-major).
 * n_leaves_out receives the leaf count n; perm [n] leaf position -> leaf index;
 * codes [n] Morton codes by leaf position; child [n-1][2] child refs (>= 0
 * internal node, else 0x80000000 | leaf index); cbox [n-1][12] child boxes;
 * root_box [6]. Any output pointer may be NULL. cap is the capacity of perm /
 * codes in elements; child/cbox must hold cap-1 nodes. */
pr_status pr_scene_read_bvh(pr_scene* scene, uint32_t level, void* stream, uint32_t cap, uint32_t* n_leaves_out,
                            uint32_t* perm, uint32_t* codes, int32_t* child, float* cbox, float* root_box);

/* Kernels enqueued by the scene's most recent pr_build_bvh and trace call. */
pr_status pr_scene_kernel_launches(const pr_scene* scene, uint32_t* build_launches, uint32_t* trace_launches);

/* Build one LBVH level over n device boxes (the device builder of
 * pr_build_bvh on caller memory; Section 2.2.3's acceleration structure,
 * here an LBVH: Morton codes of centroids, radix sort, Karras radix tree,
 * bottom-up unions). Layouts, all device memory owned by the caller:
 *   boxes     [n][6] float   lo.xyz, hi.xyz
 *   nodes     [n-1][16] float, 16-byte aligned: two child boxes and the child
 *             refs (>= 0 internal node, else 0x80000000 | box index); unused if n == 1
 *   perm      [n] uint32     sorted position -> box index
 *   codes     [n] uint32     Morton code by sorted position
 *   root_box  [8] float, 16-byte aligned: lo.xyz, 0, hi.xyz, 0
 * n <= 1024 builds in one CTA without scratch; larger n takes its scratch
 * (about 28 bytes per box) from the stream-ordered pool with cudaMallocAsync
 * and returns it with cudaFreeAsync on `stream`. Asynchronous. */
pr_status pr_lbvh_build(const float* boxes, uint32_t n, float* nodes, uint32_t* perm, uint32_t* codes,
                        float* root_box, void* stream);

/* FP32 FMA throughput probe (measurement support; no counterpart in the
 * paper): fills every SM with 256-thread CTAs, each thread running 8
 * independent fused multiply-add chains for iters rounds (1..2^24), times a
 * second launch after a warm-up with CUDA events on `stream`, and returns the
 * achieved rate in *tflops_out (2 FLOP per FMA) and the launch time in *ms_out
 * (may be NULL). It is the measured counterpart of the derived FP32 peak
 * (SMs x 128 lanes x 2 FLOP x clock) used for the trace kernel's roofline.
 * Synchronises the stream. */
pr_status pr_fma_peak_probe(uint32_t iters, float* tflops_out, float* ms_out, void* stream);

/* Largest n accepted by pr_lbvh_build_noalloc. */
#define PR_LBVH_NOALLOC_MAX_BOXES 262144u

/* pr_lbvh_build without any device allocation. The paper has no counterpart;
 * this is a service for callers that cannot let a library allocate device
 * memory while they run: applications whose device memory belongs to their own
 * allocator under a fixed budget, and latency-sensitive loops where an
 * allocation's possible synchronisation or pool growth is not acceptable.
 * Arguments, layouts and results are those of pr_lbvh_build (bit-identical).
 * Scratch comes from one fixed device array of the library (about 7.2 MB,
 * enough for PR_LBVH_NOALLOC_MAX_BOXES boxes), held until the process exits.
 * n above the limit is rejected with PR_ERR_INVALID_ARG (nothing is enqueued).
 * The array is shared by all calls and keeps the last call's contents (the
 * build clears what must start at zero); calls whose work overlaps on the GPU
 * (different streams, or different host threads, on one device) race on it
 * and must be serialised by the caller. The first call on each device, whatever
 * n, performs a one-time set-up with that device current: it looks the array
 * up, and since CUDA may load the library's modules lazily, that is when the
 * array's module is loaded and its 7.2 MB are reserved on that device if this
 * has not happened yet. Make that first call before any stream capture and
 * before any phase whose device memory must not grow. The address is kept for
 * the life of the process: cudaDeviceReset while the library is in use is not
 * supported. Later calls make no cudaMalloc, cudaFree or allocating call. */
pr_status pr_lbvh_build_noalloc(const float* boxes, uint32_t n, float* nodes, uint32_t* perm, uint32_t* codes,
                                float* root_box, void* stream);

/* ---- Batched requests (wavefront path) ---------------------------------
 * Requests of uneven size (each its own scene, camera and resolution) are
 * fused into one set of persistent kernels per bounce: a primary stage over
 * the tiles of all requests, compacted shadow and mirror ray queues, and a
 * per-pixel resolve. The per-pixel arithmetic is that of pr_trace, so each
 * request's image is bit-identical to a pr_trace of it. */
typedef struct {
  pr_scene* scene;          /* built scene */
  pr_camera camera;
  pr_trace_params params;   /* PR_TRACE_WRITE_AOV is not available in batches */
  float* out_rgba;          /* device, the whole image: height*width float4, or height*width*3
                               floats with PR_TRACE_OUTPUT_RGB in params.flags */
  uint32_t row_begin;       /* render rows [row_begin, row_begin + row_count) only; */
  uint32_t row_count;       /* row_count 0 = the whole image (row_begin must be 0) */
} pr_request;

/* Launch shape of the batched path: persistent CTAs per SM of the ray
 * stages, the primary stage's 128-pixel tile (16x8, 32x4 or 8x16) and the
 * rays a warp pops from a queue at a time (multiple of 32). megakernel = 1
 * replaces the four wavefront stages by one persistent kernel whose CTAs claim
 * 16x8 tiles of all requests and run each pixel's whole pipeline (the
 * single-request kernel's per-pixel code); megakernel = 2 runs the same with
 * one CTA per tile (ctas_per_sm unused); megakernel = 4 with one one-warp CTA
 * per 4x8 quarter of each tile (an early warp frees its slot without waiting
 * for the tile's slowest). 1, 2 and 4 need tile 16x8 and ignore
 * queue_chunk. megakernel = 3 selects the regrouped stages: traversals hand
 * their fractal (Julia, Mandelbulb) candidates on as march jobs, and a
 * persistent kernel sphere-traces them with every lane refilled from the job
 * queue as its march ends (warp ballot over the idle lanes), normals included;
 * batches of fewer than 2^31 pixels. The images are the same in every mode. */
typedef struct {
  uint32_t struct_size; /* sizeof(pr_batch_tuning) */
  uint32_t ctas_per_sm, tile_w, tile_h, queue_chunk;
  uint32_t megakernel;
} pr_batch_tuning;

typedef struct pr_batch pr_batch;

/* Allocate a batch for up to max_requests requests and max_pixels pixels in
 * total (about 310 device bytes per pixel: per-pixel state, ray queues, and
 * the regrouped mode's traversal results and march jobs). */
pr_status pr_batch_create(uint32_t max_requests, uint64_t max_pixels, pr_batch** out);

/* Set the launch shape used by later calls (PR_ERR_INVALID_ARG if unsupported). */
pr_status pr_batch_set_tuning(pr_batch* batch, const pr_batch_tuning* tuning);

/* Current launch shape of the batch. */
pr_status pr_batch_get_tuning(const pr_batch* batch, pr_batch_tuning* tuning);

/* Render n requests with direct launches on `stream` (asynchronous). The
 * request table is staged through pinned memory; a call waits until the
 * previous call's table copy has been consumed. ray_counter (device uint64,
 * optional) is incremented by the rays cast. PR_ERR_BUDGET if the pixels
 * exceed max_pixels. */
pr_status pr_trace_batch(pr_batch* batch, uint32_t n, const pr_request* requests, uint64_t* ray_counter, void* stream);

/* Same, through a CUDA graph of the stage sequence captured once per tuning
 * (the kernels read the request count and totals from device memory). */
pr_status pr_trace_batch_graph(pr_batch* batch, uint32_t n, const pr_request* requests, uint64_t* ray_counter,
                               void* stream);

/* Time every candidate launch shape on these requests (synchronises the
 * stream), keep the fastest in the batch and return it (and its time). */
pr_status pr_batch_autotune(pr_batch* batch, uint32_t n, const pr_request* requests, void* stream,
                            pr_batch_tuning* best, float* best_ms);

/* Device bytes held by the batch. */
size_t pr_batch_device_bytes(const pr_batch* batch);

/* Free the batch (synchronises the device first). */
void pr_batch_destroy(pr_batch* batch);

/* ---- Serving loop ------------------------------------------------------
 * Requests arrive at any time (pr_server_submit, thread-safe, non-blocking).
 * Scenes (inputs + BVH) stay resident in a cache keyed by scene_key; a
 * loader thread builds the scene of a request whose key is not resident, on
 * its own stream, oldest request first, once the device-memory budget holds
 * it: its device bytes are computed from the description at submit, and
 * least recently used unreferenced scenes are evicted to make room before
 * anything is allocated. A worker thread admits requests whose scene is
 * resident, in arrival order, while slots (max_active) allow, and renders.
 * PR_SERVE_CONTINUOUS: continuous batching, every iteration one batched
 * launch over row ranges of all admitted requests (at most
 * max_batch_pixels; an iteration that is a single whole request uses the
 * pr_trace megakernel, and so does the oldest request while at most
 * solo_max_waiting requests wait), so a request that arrives while others
 * are on the
 * GPU joins at the next iteration; with the batched megakernel a request is
 * complete (and pr_server_poll says so) as soon as its last tile is written,
 * through a host-mapped completion flag, not at the end of the launch.
 * PR_SERVE_PLAIN: one pr_trace per request, first come first served (the
 * comparison form; same cache and loader). Results are bit-identical to
 * pr_trace of the same request. */
#define PR_SERVE_CONTINUOUS 0u
#define PR_SERVE_PLAIN 1u

typedef struct {
  uint32_t struct_size;        /* sizeof(pr_server_config) */
  uint32_t mode;               /* PR_SERVE_CONTINUOUS or PR_SERVE_PLAIN */
  uint32_t max_active;         /* requests admitted at once */
  uint32_t solo_max_waiting;   /* PR_SERVE_CONTINUOUS: while at most this many
                                  requests wait for rows, the oldest one (if it
                                  fits max_batch_pixels) runs alone through
                                  pr_trace, as in PR_SERVE_PLAIN; 0 = always
                                  batched */
  uint64_t mem_budget_bytes;   /* device bytes for cached scenes + batch state */
  uint64_t max_batch_pixels;   /* pixels per batched iteration (>= widest image row) */
  pr_batch_tuning tuning;      /* launch shape; struct_size 0 keeps the default. Prefer
                                  megakernel 2 or 4: the persistent modes (0, 1, 3)
                                  hold every SM for a whole iteration, so scene
                                  builds on the loader's high-priority stream
                                  wait for its end */
} pr_server_config;

typedef struct {
  uint64_t scene_key;          /* equal keys share one resident scene */
  const pr_scene_desc* desc;   /* copied at submit unless scene_key is cached; may be NULL if cached */
  pr_camera camera;
  pr_trace_params params;      /* no AOV */
  float* out_rgba;             /* device, caller-owned, height*width float4 */
} pr_server_request;

/* Per-request times (seconds of a steady clock) and outcome. t_load_start /
 * t_load_end bracket the build of the request's scene (upload + BVH) when the
 * loader built it for this request, else 0. */
typedef struct {
  double t_submit, t_admit, t_first_launch, t_done;
  uint32_t status;             /* pr_status */
  uint32_t cache_hit;          /* 1 if the scene was resident at admission */
  double t_load_start, t_load_end;
} pr_request_stats;

/* cache_misses: admissions whose scene was built for them; scene_loads: scene
 * builds started by the server (equal to cache_misses unless a build failed:
 * a scene is built only once the budget holds it, so it is never built and
 * dropped again for lack of room). */
typedef struct {
  uint32_t struct_size, reserved;
  uint64_t submitted, completed, rays, iterations;
  uint64_t cache_hits, cache_misses, evictions, cache_bytes, batch_bytes;
  uint64_t scene_loads;
} pr_server_stats;

typedef struct pr_server pr_server;

/* Start a server on the current device (its worker thread and stream). */
pr_status pr_server_create(const pr_server_config* config, pr_server** out);

/* Queue a request; returns a ticket. Validates and copies the description
 * if the key is not resident. Thread-safe; does not wait for the GPU. */
pr_status pr_server_submit(pr_server* server, const pr_server_request* request, uint64_t* ticket);

/* done = 1 once the request's image is complete in out_rgba (or it failed). */
pr_status pr_server_poll(pr_server* server, uint64_t ticket, int* done, pr_request_stats* stats);

/* Wait until every submitted request is done; PR_ERR_TIMEOUT after timeout_s. */
pr_status pr_server_drain(pr_server* server, double timeout_s);

/* Totals (rays traced read from the device: synchronises the server stream). */
pr_status pr_server_get_stats(pr_server* server, pr_server_stats* stats);

/* Finish queued work, stop the worker and free everything. */
void pr_server_destroy(pr_server* server);

/* Device bytes held by the scene's arena. */
size_t pr_scene_device_bytes(const pr_scene* scene);

/* Free the scene's device memory (synchronises the device first). */
void pr_scene_destroy(pr_scene* scene);

#ifdef __cplusplus
}
#endif
#endif /* PROCEDURAY_H */
