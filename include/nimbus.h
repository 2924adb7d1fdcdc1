/*
 * nimbus.h -- C ABI of the B300 (sm_103a) point-cloud ray launcher.
 *
 * Implements the three GPU components of "A Ray Launching Approach for Computing
 * Exact Paths with Point Clouds" (arXiv 2402.13747, Section 2): voxelisation of a
 * labelled point cloud (Section 2.1), coarse path tracing by voxel cone tracing
 * (Section 2.2) and refinement of coarse paths into exact paths (Section 2.3).
 *
 * Conventions for every entry point:
 *   - Return value: NIMBUS_OK (0) or one of the NIMBUS_ERR_* codes below; a text
 *     for the last error of a context is returned by nimbus_last_error().  No
 *     C++ exception crosses this boundary and no kernel traps.
 *   - Pointers to inputs may be host or device memory (detected per pointer);
 *     inputs are copied, the caller keeps ownership.
 *   - Scenes, coarse path sets and exact path sets are owned by the library and
 *     named by opaque handles until nimbus_release().
 *   - Work is enqueued on the caller's CUDA stream (cudaStream_t passed as void*;
 *     NULL = the legacy default stream).  voxelize, trace_coarse and refine read
 *     a few counters back to size their buffers and so return after the GPU
 *     work they enqueued has finished; nimbus_query copies results to
 *     caller-owned host memory and synchronises.
 *   - Lengths in metres, angles in radians, all coordinates in one world frame.
 *   - A context is not thread-safe: serialise calls on one context.
 */
#ifndef NIMBUS_H_
#define NIMBUS_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define NIMBUS_OK 0
#define NIMBUS_ERR_ARG 1      /* invalid argument (null pointer, size, TX/RX outside the grid) */
#define NIMBUS_ERR_OOM 2      /* the context's device-memory budget or the device is exhausted */
#define NIMBUS_ERR_CUDA 3     /* a CUDA runtime error; see nimbus_last_error() */
#define NIMBUS_ERR_OVERFLOW 4 /* a bounded device buffer overflowed; sizes in nimbus_path_counts */
#define NIMBUS_ERR_TIMEOUT 5  /* a bounded device wait gave up */
#define NIMBUS_ERR_STATE 6    /* unknown handle, a handle of the wrong kind, or a failed internal self-check */
#define NIMBUS_ERR_IO 7       /* a file could not be written or read, or is not an intact scene checkpoint */

#define NIMBUS_MAX_INTERACTIONS 8 /* interactions per path, upper bound of max_int */

#if defined(__GNUC__)
#define NIMBUS_API __attribute__((visibility("default")))
#else
#define NIMBUS_API
#endif

typedef struct nimbus_ctx nimbus_ctx;
typedef uint64_t nimbus_handle;

/* Labelled point cloud (Section 2): position, normal and label per point; the
 * label is the segmentation cluster (a distinct surface).  material is carried
 * to the output (may be NULL). */
typedef struct {
  const float* xyz;         /* [n*3] positions */
  const float* nrm;         /* [n*3] unit normals */
  const uint32_t* label;    /* [n] surface labels, < 2^24 */
  const uint8_t* material;  /* [n] or NULL */
  int64_t n;
} nimbus_cloud;

/* Manually inserted diffraction edges (Section 2), exterior edges only
 * (Section 3.2): p0, p1 and the outward normals of the two faces meeting there. */
typedef struct {
  const double* edges;      /* [n*12]: p0[3] p1[3] n_face0[3] n_face1[3] */
  const uint32_t* label;    /* [n] edge labels, < 2^24 */
  int64_t n;
} nimbus_edges;

/* Voxelisation (Section 2.1) and point-set intersection (Section 2.2.1). */
typedef struct {
  double voxel_size;        /* low-resolution voxel edge h (Table 1: 0.5) */
  double sdf_sigma;         /* Gaussian width of the Eq. 1 weights */
  double sdf_eps;           /* |f| "near zero" threshold */
  double vis_ignore;        /* hits this close to a path node on its own surface are not occlusions */
  double region_min[3];     /* optional box the grid must also cover (TX/RX live inside the grid) */
  double region_max[3];
  int32_t has_region;
  int32_t dv;               /* voxel division factor D_v (Table 1: 2), 1..4 */
  int32_t sdf_max_steps;    /* steps of the |f| march */
  int32_t pad_;
} nimbus_vox_params;

/* Coarse path tracing (Section 2.2). */
typedef struct {
  double cone_half_angle;   /* constant apex half-angle alpha of every cone */
  double launch_spacing;    /* Delta of the uniform TX launch; primary half-angle max(alpha, Delta/sqrt2) */
  double sep_eps;           /* reflection separation plane offset */
  int32_t n_launch;         /* Fibonacci directions per TX (0: round(4 pi / Delta^2)) */
  int32_t max_refl;
  int32_t max_diff;
  int32_t max_int;          /* maximum interactions (Table 1: 5), <= NIMBUS_MAX_INTERACTIONS */
  int32_t kappa;            /* duplicate limit per (TX, RX, label sequence) (Table 1: 100) */
  int32_t launch_mode;      /* transmission phase (Section 2.2.2): 0 = cones on a uniform sphere grid of
                             * spacing launch_spacing; 1 = the paper's own launch, a ray from each TX toward
                             * every IE (edge IEs only when max_diff >= 1) and every RX, the visible ones
                             * becoming the initial interactions and LOS paths.  Other values: NIMBUS_ERR_ARG. */
  int64_t max_nodes;        /* bound on interaction nodes per level (0: from the memory budget) */
  int64_t max_coarse;       /* bound on coarse paths before kappa (0: from the memory budget) */
  /* Optional per-RX restrictions for batching independent requests in one call
   * (host or device arrays of n_rx, NULL = none): rx_owner[j] >= 0 lets only TX
   * rx_owner[j] reach RX j; rx_max_int[j] >= 0 keeps only coarse paths to RX j with
   * at most that many interactions.  A path with d interactions is found the same
   * way whatever the larger depth limit, so each request gets its own result. */
  const int32_t* rx_owner;
  const int32_t* rx_max_int;
} nimbus_trace_params;

/* Path refinement (Section 2.3). */
typedef struct {
  double delta;             /* convergence threshold on ||grad f|| (Table 1: 1e-4) */
  double gamma;             /* gradient-descent step scale: step = gamma / (1/a + 1/b) */
  double grad_stop;         /* iteration stops early once ||grad f|| < grad_stop */
  double freq_hz;           /* carrier frequency for the first Fresnel zone (Table 1: 60 GHz) */
  int32_t rho;              /* refinement iterations (Table 1: 2000) */
  int32_t pad_;
} nimbus_refine_params;

/* Sizes and counters of a handle (filled by nimbus_query / nimbus_query_coarse). */
typedef struct {
  int64_t n_paths;          /* exact paths after duplicate removal */
  int64_t n_refined;        /* coarse paths refined (after kappa) */
  int64_t n_refined_valid;  /* refined paths that converged and passed visibility */
  int64_t n_coarse;         /* coarse paths after the kappa limit */
  int64_t n_coarse_raw;     /* coarse paths before the kappa limit */
  int64_t n_cones;          /* cones traced (primary + every level + diffraction fans) */
  int64_t n_vis;            /* visibility rays traced during coarse tracing */
  int64_t n_nodes;          /* interaction nodes over all levels */
  int64_t needed_nodes;     /* on NIMBUS_ERR_OVERFLOW: largest level size requested */
  int64_t needed_coarse;    /* on NIMBUS_ERR_OVERFLOW: coarse paths requested */
  int64_t bytes_read;       /* algorithmic bytes of scene records read by the trace kernels */
  int32_t overflow;         /* nonzero when a bounded buffer dropped work */
  int32_t n_levels;         /* propagation levels launched */
  /* Stage kernel times in ms, measured with CUDA events on the caller's stream
   * around each stage's launches, and the algorithmic bytes each stage read. */
  double ms_vis;            /* TX -> IE / RX visibility tables */
  double ms_primary;        /* uniform launch (transmission phase) */
  double ms_levels;         /* propagation levels (voxel cone tracing) */
  double ms_kappa;          /* path expansion, grouping, sort and kappa selection */
  double ms_refine;         /* refinement kernel (Section 2.3) */
  double ms_dedup;          /* label and Fresnel duplicate removal */
  int64_t bytes_primary;
  int64_t bytes_levels;
  int64_t bytes_refine;     /* algorithmic bytes read by the refinement kernel */
  int64_t launches;         /* kernels launched by trace_coarse + refine for this handle */
  int64_t n_cones_no_rx;    /* of n_cones: last-level cones whose march was not run because it could emit
                               nothing: no RX can lie in them, or (level_rx_first) none of those that can sees
                               the apex */
} nimbus_path_counts;

/* Caller-owned host arrays for nimbus_query, each sized for n_paths entries
 * (NIMBUS_MAX_INTERACTIONS slots per path where marked [8]).  Any may be NULL. */
typedef struct {
  int32_t* tx;              /* TX index */
  int32_t* rx;              /* RX index */
  int32_t* n_int;           /* number of interactions */
  int32_t* types;           /* [8] 0 = reflection, 1 = diffraction, -1 unused */
  uint32_t* labels;         /* [8] surface / edge label per interaction */
  uint8_t* materials;       /* [8] material per interaction (255 for edges) */
  int64_t* ies;             /* [8] intersectable entity of the coarse path it came from */
  double* points;           /* [8*3] interaction points */
  double* length;           /* path length (Eq. 2) */
  double* delay;            /* length / c */
  double* grad;             /* final ||grad f|| */
  int32_t* iters;           /* refinement iterations used */
  int32_t* status;          /* 0 valid, 1 re-projection miss, 2 not converged, 3 occluded, 4 left edge */
} nimbus_path_view;

/* Caller-owned host arrays for nimbus_query_coarse, sized for n_coarse entries. */
typedef struct {
  int32_t* tx;
  int32_t* rx;
  int32_t* n_int;
  int64_t* ies;             /* [8] intersectable entities along the path */
  int32_t* types;           /* [8] */
  uint32_t* labels;         /* [8] */
  float* miss;              /* distance of the RX from the last cone's axis */
} nimbus_coarse_view;

/* Scene tables for inspection (nimbus_scene_tables), caller-owned host arrays
 * sized by nimbus_scene_info. Any may be NULL. */
typedef struct {
  int32_t* kind;            /* [n_ie] 0 point set, 1 edge segment */
  uint32_t* label;          /* [n_ie] */
  int64_t* cell;            /* [n_ie] low-resolution voxel (linear: (z*ny + y)*nx + x) */
  int32_t* gs;              /* [n_ie*3] global subvoxel coordinates */
  int64_t* prange;          /* [n_ie*2] first point (grouped order) and count */
  float* rp;                /* [n_ie*3] ray reception point */
  float* normal;            /* [n_ie*3] normalised mean normal (point IEs) */
  float* bbc;               /* [n_ie*3] bounding-box centre of the points */
  uint8_t* material;        /* [n_ie] */
  int64_t* cell_begin;      /* [n_cells] first IE of each voxel */
  int32_t* cell_count;      /* [n_cells] IEs in each voxel */
  int32_t* march;           /* [n_cells] capped L-infinity distance to the nearest voxel with IEs */
  float* slab;              /* [n_ie*4] (point IEs; zeros for edges) bounds the visibility rays use to
                               skip marches that cannot hit: smallest cosine between a point's normal
                               and the mean normal (less 1e-6), smallest and largest offset of a point
                               from the bbox centre along the mean normal, largest distance of a point
                               from that centre */
} nimbus_scene_view;

/* Contexts (operational; the paper has no counterpart).
 * nimbus_create: a context on CUDA device `device` with a device-memory budget in
 * bytes (0 = 90% of the free memory); *out receives it, owned by the caller until
 * nimbus_destroy.  NIMBUS_ERR_ARG for a NULL out or a device index this machine does
 * not have (then *out = NULL); NIMBUS_ERR_CUDA when the device cannot be queried.
 * nimbus_destroy: releases every scene, coarse set and path set of the context,
 * synchronises its device and frees the context; NIMBUS_ERR_ARG for NULL.
 * nimbus_last_error: the text of the context's last error, valid until the next call
 * on that context ("null context" for NULL). */
NIMBUS_API int nimbus_create(nimbus_ctx** out, int device, size_t mem_budget_bytes);
NIMBUS_API int nimbus_destroy(nimbus_ctx* ctx);
NIMBUS_API const char* nimbus_last_error(nimbus_ctx* ctx);

/* Section 2.1: bin the cloud into subvoxels (h / D_v) by a sort on the
 * (voxel, subvoxel, kind, label) key, build one intersectable entity per
 * (subvoxel, label) point group (reception point = centroid, normal =
 * normalised mean normal) and per edge segment inside a subvoxel, give each
 * voxel its entity range and compute the march distance field of
 * Section 2.2.4.  edges may be NULL.  scene_out receives the scene handle. */
NIMBUS_API int nimbus_voxelize(nimbus_ctx* ctx, const nimbus_cloud* cloud, const nimbus_edges* edges,
                    const nimbus_vox_params* params, nimbus_handle* scene_out, void* stream);

/* Dynamic scenes (the paper treats static clouds; the tables rebuilt are those of
 * Section 2.1): drop the points of the scene whose position lies inside the box
 * [aabb_min, aabb_max] (metres, world frame) and add `replacement` (host or device
 * arrays, copied; may be NULL or empty), then rebuild the scene's tables in place on
 * the same grid.  The result equals a full nimbus_voxelize of the updated cloud on
 * that grid.  NIMBUS_ERR_ARG for a NULL box, NIMBUS_ERR_STATE for a handle that is
 * not a scene of ctx, NIMBUS_ERR_OOM past the budget. */
NIMBUS_API int nimbus_update_region(nimbus_ctx* ctx, nimbus_handle scene, const double aabb_min[3],
                         const double aabb_max[3], const nimbus_cloud* replacement, void* stream);

/* Section 2.2: for every TX, a uniform launch of cones on a Fibonacci lattice
 * (transmission phase), then level by level reflected cones and Keller-cone
 * diffraction fans (propagation phase) traversed by voxel cone tracing;
 * cone-sphere tests, separation planes and visibility rays decide which
 * entities a cone reaches, RXs reached give coarse paths, and at most kappa
 * coarse paths are kept per (TX, RX, label sequence).  tx [n_tx*3], rx [n_rx*3]
 * (host or device).  coarse_out receives the coarse set handle.  A cone of the last
 * depth that no RX can lie in, or (level_rx_first) none of whose reachable RXs sees
 * its apex, produces nothing, so it is counted but not marched
 * (nimbus_path_counts.n_cones_no_rx).  Errors: NIMBUS_ERR_ARG for bad parameters or
 * a TX/RX outside the grid; NIMBUS_ERR_OVERFLOW with the needed bounds in the counts
 * (the handle is still returned); NIMBUS_ERR_TIMEOUT when a bounded device wait of the
 * propagation gave up; NIMBUS_ERR_STATE when a self-check of the propagation's
 * indices failed (never expected; the message names the check and its values);
 * NIMBUS_ERR_OOM past the budget. */
NIMBUS_API int nimbus_trace_coarse(nimbus_ctx* ctx, nimbus_handle scene, const double* tx, int32_t n_tx,
                        const double* rx, int32_t n_rx, const nimbus_trace_params* params,
                        nimbus_handle* coarse_out, void* stream);

/* Section 2.3: refine every coarse path by gradient descent on the path length
 * (Eq. 2) over the local variables (r, s) of reflections and t of
 * diffractions, re-projecting reflection points onto the point cloud by a ray,
 * for rho iterations or until ||grad f|| < grad_stop; keep paths with
 * ||grad f|| < delta whose segments are all visible; remove duplicates by label
 * sequence (shortest kept) and by first Fresnel zone (delay order).
 * paths_out receives the exact path set handle. */
NIMBUS_API int nimbus_refine(nimbus_ctx* ctx, nimbus_handle scene, nimbus_handle coarse,
                  const nimbus_refine_params* params, nimbus_handle* paths_out, void* stream);

/* The exact paths of Section 2.3 (per path: TX and RX index, interaction types,
 * labels, materials and entities, FP64 interaction points, length, delay = length /
 * c, final gradient norm, iterations and status; layouts in nimbus_path_view):
 * counts (required) and, when view != NULL, the paths copied into the caller's host
 * arrays, sized from a call with view == NULL.  which = 0: paths after duplicate
 * removal, in delay order; 1: every refined coarse path with its status.
 * Synchronises the stream.  NIMBUS_ERR_ARG for a NULL counts, NIMBUS_ERR_STATE for
 * a handle that is not a path set of ctx. */
NIMBUS_API int nimbus_query(nimbus_ctx* ctx, nimbus_handle paths, int32_t which, nimbus_path_counts* counts,
                 const nimbus_path_view* view, void* stream);

/* The coarse paths of Section 2.2.3 after the kappa limit (TX, RX, interaction
 * entities, types and labels, miss distance of the last cone axis from the RX;
 * layouts in nimbus_coarse_view): counts (required) and, when view != NULL, the paths
 * copied into the caller's host arrays.  Synchronises the stream.  NIMBUS_ERR_ARG for
 * a NULL counts, NIMBUS_ERR_STATE for a handle that is not a coarse set of ctx. */
NIMBUS_API int nimbus_query_coarse(nimbus_ctx* ctx, nimbus_handle coarse, nimbus_path_counts* counts,
                        const nimbus_coarse_view* view, void* stream);

/* Grid and table sizes of a scene (Section 2.1): origin[3] in metres, dims[3] in
 * voxels, the number of entities and of grouped points; any output may be NULL.
 * NIMBUS_ERR_STATE for a handle that is not a scene of ctx. */
NIMBUS_API int nimbus_scene_info(nimbus_ctx* ctx, nimbus_handle scene, double origin[3], int32_t dims[3],
                      int64_t* n_ie, int64_t* n_points);

/* Copy a scene's entity and voxel tables (Section 2.1; layouts in
 * nimbus_scene_view, sized by nimbus_scene_info) into caller-owned host arrays.
 * Synchronises the stream.  NIMBUS_ERR_ARG for a NULL view, NIMBUS_ERR_STATE for a
 * handle that is not a scene of ctx. */
NIMBUS_API int nimbus_scene_tables(nimbus_ctx* ctx, nimbus_handle scene, const nimbus_scene_view* view,
                        void* stream);

/* Free a scene, coarse set or path set (operational; the paper has no counterpart).
 * NIMBUS_ERR_STATE for a handle ctx does not hold. */
NIMBUS_API int nimbus_release(nimbus_ctx* ctx, nimbus_handle h);

/* Bytes of device memory the context currently holds (operational; the paper has no
 * counterpart).  NIMBUS_ERR_ARG for a NULL argument. */
NIMBUS_API int nimbus_memory_used(nimbus_ctx* ctx, size_t* bytes);

/* Number of CUDA kernels this library has launched in this process so far (all
 * contexts); differences around a region count the kernels launched in it
 * (operational; the paper has no counterpart).  NIMBUS_ERR_ARG for NULL. */
NIMBUS_API int nimbus_kernel_launches(int64_t* count);

/* Number of device allocations (cudaMallocAsync calls) this library has made in this
 * process so far (all contexts); differences around a call count the allocations it
 * made (operational; the paper has no counterpart).  NIMBUS_ERR_ARG for NULL. */
NIMBUS_API int nimbus_device_allocations(int64_t* count);

/* ---------------------------------------------------------------------------
 * Scene checkpoint.
 *
 * Not part of the paper's method: persistence for a serving process.
 * nimbus_scene_save writes the scene's current cloud (after any region updates), its
 * edges, voxelisation parameters and grid to `path`.  nimbus_scene_load reads such a
 * file into a new scene of `ctx` (any device); its derived tables are rebuilt on the
 * saved grid, so they equal those of the saved scene bit for bit.  Both synchronise
 * `stream`.  File: little-endian, magic "NIMBUSC1", version 1, FNV-1a checksum of the
 * payload; a file that cannot be opened, is truncated, foreign or damaged returns
 * NIMBUS_ERR_IO and creates nothing.
 */
NIMBUS_API int nimbus_scene_save(nimbus_ctx* ctx, nimbus_handle scene, const char* path, void* stream);
NIMBUS_API int nimbus_scene_load(nimbus_ctx* ctx, const char* path, nimbus_handle* scene_out, void* stream);

/* ---------------------------------------------------------------------------
 * Automatic labels and exterior edges for an unlabelled cloud.
 *
 * The method takes a labelled cloud whose labels are the clusters of a segmentation
 * into distinct surfaces, and diffraction edges inserted by hand (Section 2; the
 * experiments of Section 3 labelled with a plane-fitting algorithm from PCL, and raw
 * sensor clouds are left to future work).  nimbus_segment produces both from positions
 * and normals alone, by this reading:
 *  1. the points are binned into subvoxels exactly as nimbus_voxelize bins them
 *     (Section 2.1); the points of one subvoxel, in input order, form a group;
 *  2. each group gets an FP64 centroid, covariance and plane normal (the eigenvector of
 *     the smallest eigenvalue, turned to agree with the sum of the input normals); it is
 *     planar when it has >= min_points points, a positive trace, smallest eigenvalue
 *     <= flat_max * trace and middle eigenvalue >= spread_min * trace;
 *  3. planar groups in 26-adjacent subvoxels are joined when their normals agree
 *     (n_a . n_b >= cos join_angle) and each centroid is within join_dist of the other's
 *     plane; connected groups form one surface, a non-planar group a surface of its
 *     own; surfaces are numbered in the order of their first group in (voxel, subvoxel)
 *     order;
 *  4. a point takes its group's surface when that group is planar, agrees with the
 *     point's normal (>= cos join_angle) and has the point within join_dist of its
 *     plane; otherwise the surface of the nearest such planar neighbour group (ties: the
 *     lower group); otherwise its group's surface;
 *  5. two surfaces with >= edge_min_groups planar groups each, meeting in 26-adjacent
 *     subvoxels, form an exterior edge when their planes (pooled FP64 moments of their
 *     planar groups) are >= edge_angle apart and each centroid lies behind the other's
 *     plane.  The edge lies on the planes' intersection line, at its point nearest the
 *     mean centroid of the meeting groups, spans those centroids' projections, and
 *     carries the two planes' normals as face normals.  Edges are ordered by their
 *     surface pair; edge e has label n_surfaces + e.
 * The outputs feed nimbus_voxelize directly (labels as the cloud's labels, edges as
 * nimbus_edges). */
typedef struct {
  double voxel_size;        /* the voxelisation grid (Table 1: 0.5) */
  double flat_max;          /* planarity: smallest covariance eigenvalue <= flat_max * trace (0.02) */
  double spread_min;        /* ... and middle eigenvalue >= spread_min * trace (0.05): not a row of points */
  double join_angle;        /* radians: largest angle between the normals of joined groups (10 deg) */
  double join_dist;         /* metres: largest centroid-to-plane offset of joined groups and fitted points (0.03) */
  double edge_angle;        /* radians: smallest angle between the planes of an exterior edge (30 deg) */
  int32_t dv;               /* voxel division factor D_v (Table 1: 2), 1..4 */
  int32_t min_points;       /* fewest points of a planar group (3), >= 3 */
  int32_t edge_min_groups;  /* fewest planar groups of each surface of an edge (4), >= 1 */
  int32_t pad_;
} nimbus_segment_params;

typedef struct {
  int64_t n_groups;         /* occupied subvoxels */
  int64_t n_planar;         /* planar groups */
  int64_t n_surfaces;       /* surfaces: point labels are < n_surfaces (a non-planar group whose points
                               all went to neighbours keeps an empty label) */
  int64_t n_edges;          /* exterior edges found (labels n_surfaces .. n_surfaces + n_edges - 1) */
  double ms;                /* device time of steps 2-5 */
  double ms_total;          /* device time of the call, including the binning voxelisation */
} nimbus_segment_counts;

/* Labels and exterior edges of an unlabelled cloud (cloud->label and ->material are
 * ignored).  labels: [cloud->n] out; edges: [edges_cap * 12] out as p0 p1 n_face0
 * n_face1; edge_labels: [edges_cap] out; any of them host or device memory, owned by
 * the caller (edges and edge_labels may be NULL when edges_cap is 0).  counts is always
 * filled on success and on NIMBUS_ERR_OVERFLOW, which means more than edges_cap edges
 * exist: the first edges_cap are written and counts->n_edges says how many to allow.
 * An empty cloud or out-of-range parameter is NIMBUS_ERR_ARG; a union-find step bound
 * reached (not expected) is NIMBUS_ERR_TIMEOUT.  Synchronises `stream`. */
NIMBUS_API int nimbus_segment(nimbus_ctx* ctx, const nimbus_cloud* cloud, const nimbus_segment_params* params,
                              uint32_t* labels, double* edges, uint32_t* edge_labels, int64_t edges_cap,
                              nimbus_segment_counts* counts, void* stream);

/* ---------------------------------------------------------------------------
 * Launch configuration and autotuner.
 *
 * Not part of the paper's method: how the kernels are laid out on the GPU, never what
 * they compute.  Every setting gives bit-identical results; only the time changes.
 */
typedef struct {
  int32_t level_block;      /* threads per block of the propagation levels: 128, 256 or 512 */
  int32_t refine_blocks;    /* 4-warp refinement blocks per SM: 1..8 (at most as many as fit), 0 = as many as fit */
  int32_t refine_order;     /* 1: refine the paths with the most interactions first; 2: first the paths whose
                               re-projection rays graze their surfaces at the start (smallest |n . d|), then by
                               interactions; 0: in coarse order */
  int32_t graph;            /* 1: each stretch of a call with no host round trip (trace: RX table, march field,
                               transmission phase and all depths; refine: refinement, final visibility and
                               winners; then dedup) is captured on a private stream and launched on the
                               caller's stream as one CUDA graph; 0: the same launches issued directly */
  double level_ms;          /* after nimbus_autotune: time of the chosen level layout on the sample, else 0 */
  double refine_ms;         /* after nimbus_autotune: time of the chosen refinement layout on the sample, else 0 */
  int32_t level_queue;      /* 1: all propagation depths in one launch, a cone of depth d + 1 starting as soon as
                               its parent emitted it (waits bounded; NIMBUS_ERR_TIMEOUT if one gives up);
                               0: one launch per depth */
  int32_t refine_split;     /* > 0: refine in two launches, the first stopping every path after this many
                               iterations and the second resuming the unfinished ones, costliest per
                               iteration first (0..65535; 0 or >= rho: one launch) */
  int32_t refine_split_key; /* the second launch's order: 0 the cost per iteration so far; 1 the predicted
                               remaining time (that cost x the iterations still needed at the gradient's
                               rate of decrease over the second half of the first launch) */
  int32_t level_help;       /* one launch per depth only: 1, a warp whose cones are done walks visibility rays
                               of the cones still running in its block (the candidates of an evaluation wait in
                               a shared-memory list); 0, every warp walks only its own cones' rays */
  int32_t level_rx_first;   /* 1: at the last depth, a cone none of whose reachable RXs sees its apex is not
                               marched (it could emit nothing); pays where few reachable RXs are visible */
} nimbus_tuning;

/* The context's launch configuration (defaults 512, 0, 1, 1, level_queue 0, refine_split 0,
 * refine_split_key 0, level_help 1, level_rx_first 1). */
NIMBUS_API int nimbus_get_tuning(nimbus_ctx* ctx, nimbus_tuning* out);

/* Replace it.  A value out of range returns NIMBUS_ERR_ARG and changes nothing. */
NIMBUS_API int nimbus_set_tuning(nimbus_ctx* ctx, const nimbus_tuning* t);

/* Testing the bounded waits.  Every device wait of the propagation levels (a warp of
 * the single launch waiting for a task or a record, a cone waiting for the visibility
 * rays other warps took, a warp waiting for the cones of its block) gives up after a
 * limit in SM clock cycles: seconds by default.  This sets that limit for the
 * context's later trace calls (`cycles` > 0), or restores the defaults (0).  With a
 * limit of a few cycles the waits give up at once: the call then returns
 * NIMBUS_ERR_TIMEOUT and frees what it allocated, and the context stays usable.
 * Negative values return NIMBUS_ERR_ARG. */
NIMBUS_API int nimbus_set_wait_limit(nimbus_ctx* ctx, int64_t cycles);

/* Autotuner.  Traces the given TX/RX set on `scene` once per level layout (blocks of
 * 128, 256 or 512 threads x one launch per depth, with or without idle warps walking
 * other warps' visibility rays, or one launch for all depths) and keeps the fastest
 * propagation time; then it tries the last depth's RX visibility test the other way.  Then it refines that coarse set once per refinement layout with
 * all resident blocks per SM: one launch in coarse order, most interactions first or
 * grazing rays first; and two launches, the first in coarse order or most interactions
 * first and stopping at 64, 128 or 512 iterations, the second in either of its orders;
 * it keeps the fastest.  The result is stored in the context for the calls that follow
 * and written to `out` (may be NULL).  Every layout gives the same results; tune on the
 * workload itself where its refinement ends on long paths (a small sample is one tail
 * whatever the layout).  Times are CUDA events on `stream`; the call synchronises.
 * Errors of the trace or refinement (including NIMBUS_ERR_OVERFLOW: the set needs
 * larger bounds) are returned unchanged and leave the configuration as it was. */
NIMBUS_API int nimbus_autotune(nimbus_ctx* ctx, nimbus_handle scene, const double* tx, int32_t n_tx,
                               const double* rx, int32_t n_rx, const nimbus_trace_params* trace_params,
                               const nimbus_refine_params* refine_params, nimbus_tuning* out, void* stream);

/* ---------------------------------------------------------------------------
 * Voxelisation without any device allocation.
 *
 * Not part of the paper's method (the paper has no counterpart): an operational
 * variant for callers that cannot allocate device memory while they run -- for
 * example a process whose device memory is carved up in advance by another
 * allocator, or a real-time loop that must not block on the allocator.  It computes the same tables as
 * nimbus_voxelize + nimbus_scene_tables for a cloud without edges, but writes them
 * into caller-owned device buffers and keeps every intermediate in one fixed
 * device array inside this library (NIMBUS_STATIC_MAX_POINTS points and
 * NIMBUS_STATIC_MAX_CELLS voxels at most; about 35 MB that every GPU which loads
 * the library holds until the process exits).
 *
 * - Inputs (cloud->xyz, nrm, label, material) must be device pointers.
 * - Larger clouds or grids: NIMBUS_ERR_ARG with a message; output capacities
 *   too small: NIMBUS_ERR_OVERFLOW with the needed sizes in *info, and the
 *   outputs untouched.  A voxel capacity below the grid's size is found before
 *   the entities are counted: info->n_cells is set and info->n_ie is -1.
 * - The first call on a device resolves the fixed array's device address
 *   (cudaGetSymbolAddress) with that device current; make that first call before
 *   any stream capture on that device.
 * - Every call shares the one array: calls that overlap on the GPU (other
 *   streams, other host threads) race and must be serialised by the caller.  The
 *   call reads two counters back and so returns after its work has finished; it
 *   synchronises its stream, so it cannot run inside a CUDA host function (one
 *   that cudaLaunchHostFunc or a graph host node runs) or under stream capture.
 * - Null or non-device output pointers for a non-zero capacity: NIMBUS_ERR_ARG,
 *   before any device work.
 * - Calls no cudaMalloc, cudaFree or other allocating routine. */
#define NIMBUS_STATIC_MAX_POINTS (1 << 17)
#define NIMBUS_STATIC_MAX_CELLS (1 << 20)

typedef struct {          /* caller-owned device buffers */
  int32_t* kind;          /* [ie_capacity] 0 point set (edges are not taken) */
  uint32_t* label;        /* [ie_capacity] */
  int32_t* gs;            /* [ie_capacity*3] global subvoxel coordinates */
  int32_t* pcount;        /* [ie_capacity] points in the entity */
  float* rp;              /* [ie_capacity*3] reception point (centroid) */
  float* normal;          /* [ie_capacity*3] normalised mean normal */
  float* bbc;             /* [ie_capacity*3] bounding-box centre */
  uint8_t* material;      /* [ie_capacity] */
  int64_t ie_capacity;
  uint32_t* cell_begin;   /* [cell_capacity] first entity of each voxel (0 when empty) */
  uint32_t* cell_count;   /* [cell_capacity] */
  uint8_t* march;         /* [cell_capacity] capped L-infinity distance to a voxel with entities */
  int64_t cell_capacity;
} nimbus_static_tables;

typedef struct {          /* host outputs */
  double origin[3];
  int32_t dims[3];
  int32_t pad_;
  int64_t n_ie;
  int64_t n_cells;
} nimbus_static_info;

NIMBUS_API int nimbus_voxelize_static(nimbus_ctx* ctx, const nimbus_cloud* cloud, const nimbus_vox_params* params,
                                      const nimbus_static_tables* out, nimbus_static_info* info, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* NIMBUS_H_ */
