/*
 * grtx.h -- C ABI of libgrtx.so, a GB300 (sm_103a) Gaussian ray tracer after GRTX
 * (arXiv 2601.20429): every anisotropic Gaussian is a unit sphere in its own instance space
 * (Sec. IV-A), rays traverse an LBVH whose leaves are those instances, and tracing runs in
 * rounds that gather the k nearest hits in a k-buffer (Sec. III-A), composite them front to
 * back with early termination (Sec. II-B Eq. volume-render, Sec. III-A), and resume the next
 * round from checkpointed nodes and evicted hits instead of the root (Sec. IV-B, Listing 1).
 *
 * Conventions for every entry point:
 *   - Pointers named d_* or documented as "device" point to device memory on the current
 *     CUDA device; the caller owns them unless stated. Host structs are read during the call
 *     only and may be freed when it returns.
 *   - All work is enqueued on the given stream (a cudaStream_t passed as void*, NULL = the
 *     legacy default stream) and is asynchronous unless stated. Outputs are valid once the
 *     stream reaches the point after the call.
 *   - Every call returns a grtx_status. No exception or longjmp crosses the ABI. Argument
 *     errors are detected on the host before anything is enqueued. Device-side capacity
 *     overflows are never fatal: the affected ray falls back to restarting from the root
 *     (always correct) and the event is counted in grtx_stats.
 *   - Floating point is IEEE FP32 throughout; arrays are C-contiguous structure-of-arrays.
 *   - A scene or server may be used from one host thread at a time. The traces of one scene
 *     share its per-slot workspace and queue counters, so they must be ordered: issue them
 *     on one stream, or synchronise between streams. Different scenes may trace
 *     concurrently.
 */
#ifndef GRTX_H
#define GRTX_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define GRTX_API __attribute__((visibility("default")))
#define GRTX_VERSION 1
#define GRTX_DEFAULT_CKPT_CAPACITY 256
#define GRTX_DEFAULT_SINGLE_CAPACITY 2048
#define GRTX_DEFAULT_EVICT_CAPACITY 512

/* ---------------------------------------------------------------------------------------- */
/* Status codes                                                                             */
/* ---------------------------------------------------------------------------------------- */
typedef enum grtx_status {
    GRTX_OK = 0,
    GRTX_ERR_INVALID_ARG = 1,     /* a pointer, size or parameter is out of its documented range */
    GRTX_ERR_OOM = 2,             /* a device allocation failed                                 */
    GRTX_ERR_CUDA = 3,            /* a CUDA runtime call failed (sticky device error, launch)  */
    GRTX_ERR_OVERFLOW_FATAL = 4,  /* a fixed limit was exceeded with no fallback (BVH depth)   */
    GRTX_ERR_TIMEOUT = 5,         /* a bounded wait ran out                                    */
    GRTX_ERR_BUSY = 6,            /* the server has no free slot or memory for the request     */
    GRTX_ERR_NOT_FOUND = 7        /* an id (scene, request) is unknown                          */
} grtx_status;

/* ---------------------------------------------------------------------------------------- */
/* Plain data types                                                                         */
/* ---------------------------------------------------------------------------------------- */

/* Raw Gaussian parameters (Sec. II-B: mean, covariance from rotation and scale, opacity,
 * SH coefficients). All device pointers, caller-owned, FP32:
 *   means [n][3]; log_scales [n][3] (s = exp); quats [n][4] as (w,x,y,z), any non-zero length
 *   (normalised inside); opacity_logits [n] (o = sigmoid); sh [n][(L+1)^2][3], L = sh_degree. */
typedef struct grtx_gaussians {
    const float *means;
    const float *log_scales;
    const float *quats;
    const float *opacity_logits;
    const float *sh;
    int64_t n;
    int32_t sh_degree;           /* 0..3 */
    int32_t reserved;
} grtx_gaussians;

/* Gradients w.r.t. the raw parameters, same shapes as grtx_gaussians, device, caller-owned.
 * grtx_trace_backward ADDS into them (the caller zeroes them first). A NULL member skips
 * that parameter. */
typedef struct grtx_grads {
    float *means;
    float *log_scales;
    float *quats;
    float *opacity_logits;
    float *sh;
} grtx_grads;

enum { GRTX_FORM_SPHERE = 0,        /* one leaf per Gaussian, analytic unit sphere (Sec. IV-A) */
       GRTX_FORM_PROXY20 = 1,       /* one leaf per proxy triangle: 20-triangle icosahedron
                                       around each Gaussian, monolithic BVH (Sec. III-C Obs. I) */
       GRTX_FORM_ICO20 = 2,         /* two-level: the sphere form's BVH over Gaussian instances,
                                       and one shared template BVH of a 20-triangle icosahedron
                                       around the unit sphere (Sec. IV-A, second option) */
       GRTX_FORM_ICO80 = 3 };       /* as ICO20 with the 80-triangle icosphere */
enum { GRTX_TRAVERSAL_CHECKPOINT = 0, /* resume from checkpointed nodes + eviction list (IV-B) */
       GRTX_TRAVERSAL_RESTART = 1,    /* restart from the root every round (Sec. III-A)       */
       GRTX_TRAVERSAL_SINGLE = 2 };   /* one traversal collecting every hit, then sort and
                                         blend (single-round baseline, Sec. III-C Obs. II)   */

/* Tracing parameters. k: k-buffer size, one of 1, 2, 4, 8, 16, 32 (Sec. III-A).
 * alpha_min: a Gaussian is hit where its response reaches alpha_min (0.01); it also sets the
 * ellipsoid radius kappa = sqrt(2 ln(o / alpha_min)) used at build time. T_min: a ray stops
 * right after the Gaussian that takes its transmittance below T_min (1e-3). alpha_max: clamp
 * on alpha before compositing (0.99). bg: background colour added as T * bg.
 * ckpt_capacity / evict_capacity: checkpoint and eviction entries per resident ray slot
 * (Sec. IV-B "Checkpoint and Eviction Buffer"); 0 selects GRTX_DEFAULT_CKPT_CAPACITY (256)
 * and GRTX_DEFAULT_EVICT_CAPACITY (512). A ray whose list overflows redoes that round from
 * the root and restarts from then on (exact; counted in fallbacks); on deep scenes such rays
 * hold their launch long after the others finish, so the defaults leave room for the deep
 * views of the configurations (a 6M-Gaussian outdoor frame had 24,610 such rays with 128
 * eviction entries, none with 512). With GRTX_TRAVERSAL_SINGLE, ckpt_capacity is the
 * number of hits a ray slot's list holds (0 selects GRTX_DEFAULT_SINGLE_CAPACITY, 2048, the
 * top of the paper's 512-2048); a ray with more hits is traced with k-buffer rounds
 * restarted from the root instead (same result, counted in fallbacks), and k must still be
 * one of the valid sizes.
 * traversal: GRTX_TRAVERSAL_*, for either form: {sphere, proxy} x {checkpoint, restart} are the
 * paper's GRTX, GRTX-HW only (proxy + checkpoint), GRTX-SW only (sphere + restart) and the
 * baseline (proxy + restart) of Sec. V-B.
 * bvh_codes (read by grtx_build_bvh only): the sort key of the build, GRTX_CODES_SIZED (0,
 * the default: grtx_morton_codes_sized) or GRTX_CODES_CENTROID (grtx_morton_codes).
 * bvh_builder (read by grtx_build_bvh only): GRTX_BUILDER_PLOC (0, the default: clustering
 * of the sorted leaves, grtx_ploc_tree) or GRTX_BUILDER_LBVH (the binary radix tree of the
 * codes, grtx_radix_tree). The tree shape changes the cost of a trace, never its result.
 * packet_stack: entries of the per-warp stack that a warp-packet traversal may use (0: all
 * GRTX_PACKET_STACK); a packet that would need more falls back to tracing its rays one by
 * one, with the same result. Smaller values exist to exercise that fallback. (The stack holds
 * the far children still pending along the warp's path: 48 entries of 16 bytes per warp, so
 * that with the k-buffer a 128-ray block takes 19 KB of shared memory, and 8 blocks leave
 * the SM a 92 KB L1 instead of 60 KB; no packet overflowed it on the 111-level tree of the
 * 6M outdoor scene.)
 * bvh_width (the paper traverses a 6-wide BVH, Sec. V-A): 0 or 2, binary nodes; 4, the build
 * of a sphere-form scene also collapses the binary tree into 4-wide nodes (each binary node at
 * even depth becomes a node over its grandchildren, 128 bytes: lo x, lo y, lo z, hi x, hi y,
 * hi z of the four children as float4 rows, then the four child refs, then padding), and
 * grtx_trace_forward with bvh_width 4 traverses them (checkpoint or restart traversal, no
 * saved lists; GRTX_ERR_INVALID_ARG on a scene built without them). Every other entry point
 * traverses the binary nodes. The image does not depend on the width.
 * bvh_quantize (read by grtx_build_bvh with bvh_width 4): 1 stores the 4-wide nodes with
 * quantised child boxes in 64 bytes: the node's lower corner (3 floats) and a power-of-two
 * step per axis, then per child and axis an 8-bit lower and upper grid coordinate, rounded
 * outwards so that the decoded box (corner + q * step, one FMA) contains the child's box;
 * then the four child refs. A trace reads whichever format the scene was built with. */
#define GRTX_PACKET_STACK 48
enum { GRTX_CODES_SIZED = 0, GRTX_CODES_CENTROID = 1 };
enum { GRTX_BUILDER_PLOC = 0, GRTX_BUILDER_LBVH = 1 };
#define GRTX_PLOC_RADIUS 16
typedef struct grtx_params {
    int32_t k;
    int32_t traversal;
    float alpha_min;
    float T_min;
    float alpha_max;
    float bg[3];
    int32_t ckpt_capacity;
    int32_t evict_capacity;
    int32_t bvh_codes;
    int32_t bvh_builder;
    int32_t packet_stack;
    int32_t bvh_width;
    int32_t bvh_quantize;
} grtx_params;

enum { GRTX_CAMERA_PINHOLE = 0, GRTX_CAMERA_FISHEYE = 1, GRTX_CAMERA_RAYS = 2 };

/* A camera (rays generated in-kernel) or an explicit ray list.
 * Pinhole: pixel (x, y), y = 0 the top row, has direction
 *   normalize(forward + u right + v up), u = (2(x+.5)/W - 1) tan(fov/2) W/H,
 *   v = (1 - 2(y+.5)/H) tan(fov/2); fov is the vertical field of view in radians.
 * Fisheye (equidistant): the angle from forward is r / f with r the distance in pixels of
 *   the pixel centre from the image centre and f = (W/2) / fov, i.e. fov is the angle
 *   reached at half the image width.
 * Rays: width*height rays (height may be 1) from device arrays ray_origins [n][3],
 *   ray_dirs [n][3] (any non-zero length; t is measured in units of |dir|), and optional
 *   ray_tnear / ray_tfar [n] (NULL: the scalar t_near / t_far below). A list of at least
 *   four rows is taken as an image and traced in 8x4 tiles, like a camera, so that a warp's
 *   rays are neighbours; the output order is the same either way.
 * Every ray accepts hits with t_near < t <= t_far. Output pixel index = y * width + x. */
typedef struct grtx_camera {
    int32_t type;
    int32_t width, height;
    float pos[3], right[3], up[3], forward[3];
    float fov;
    float t_near, t_far;
    const float *ray_origins;
    const float *ray_dirs;
    const float *ray_tnear;
    const float *ray_tfar;
} grtx_camera;

/* Device counters, summed (+=) over rays by the trace calls when a grtx_stats* is given.
 * nodes: internal BVH nodes fetched; leaves: leaf records tested (Gaussians or triangles);
 * blended: Gaussians composited; rounds: tracing rounds; ckpt_writes: checkpoint entries
 * written; evictions: entries written to the eviction list; fallbacks: rays that exceeded a
 * capacity and restarted from the root; stack_overflow: traversal stack overflows (never
 * expected: the build rejects trees deeper than the stack); collected: hits appended to the
 * single-round lists (GRTX_TRAVERSAL_SINGLE only); bounds_errors: node, leaf-record or
 * Gaussian indices that the traversal met outside the scene's arrays. The kernels that fill
 * these counters compare each such index with its array's size before the fetch, count one
 * outside and skip it (never expected: every index comes from the scene's own build). */
typedef struct grtx_stats {
    unsigned long long rays, nodes, leaves, blended, rounds, ckpt_writes, evictions, fallbacks,
        stack_overflow, collected, bounds_errors;
} grtx_stats;

/* Blend lists a forward trace saves for its backward (grtx_trace_backward_saved): for each
 * ray, the leaf slots it blended, in blend order. leaves: device [n_rays][cap]; n: device
 * [n_rays], the number blended; a count above cap means the list is incomplete, and the
 * backward replays that ray's rounds. Leaf slots index the scene's leaf order: the lists
 * hold while the scene is not updated; an entry at or past the scene's number of valid
 * Gaussians (a list from another scene) is skipped, never read. Caller-owned device memory. */
typedef struct grtx_saved {
    uint32_t *leaves;
    int32_t *n;
    int32_t cap;
    int32_t reserved;
} grtx_saved;

/* Outputs of a forward trace. rgbT: device [n_rays][4] = (C + T bg, T), required.
 * n_blended: optional device [n_rays], Gaussians composited per ray. blended_ids: optional
 * device [n_rays][ids_cap], the first ids_cap composited Gaussian ids per ray in blend order
 * (unused tail entries are 0xFFFFFFFF). stats: optional device grtx_stats (accumulated).
 * visits / visits_n: optional node-visit log of sampled rays, for counting total against
 * distinct node fetches (a revisit is a fetch of a node the ray fetched before, the work
 * checkpointing removes, Sec. III-C). A ray with output index p is logged when
 * p % visits_stride == 0 and p / visits_stride < visits_rows: row r = p / visits_stride of
 * device [visits_rows][visits_cap] receives its fetches in order (internal node index, or
 * GRTX_LEAF | leaf index for a leaf record; the nodes of an icosphere template are not
 * logged), and visits_n[r] their number, which may exceed visits_cap (the row then holds the
 * first visits_cap). Rows of rays that are not traced keep their contents; visits_n is
 * zeroed by the call. Both pointers or neither; cap, stride and rows >= 1 when given.
 * saved: optional blend lists for the backward (sphere form, checkpoint or restart
 * traversal, with no other optional output: the saving forward is its own uninstrumented
 * kernel). With any other optional output requested the kernel takes a slower instrumented
 * path. */
typedef struct grtx_trace_outputs {
    float *rgbT;
    int32_t *n_blended;
    uint32_t *blended_ids;
    int32_t ids_cap;
    int32_t reserved;
    grtx_stats *stats;
    uint32_t *visits;
    uint32_t *visits_n;
    int32_t visits_cap, visits_stride, visits_rows, reserved2;
    const grtx_saved *saved;
} grtx_trace_outputs;

/* Host-readable description of a built scene. */
typedef struct grtx_scene_info {
    int64_t n_gaussians;       /* n given to the build                                     */
    int64_t n_valid;           /* Gaussians with o > alpha_min, i.e. in the BVH            */
    int64_t n_leaves;          /* BVH leaves: n_valid (sphere) or 20 n_valid (proxy)        */
    int64_t n_nodes;           /* internal BVH nodes (n_leaves - 1, at least 1)             */
    int32_t depth;             /* deepest leaf, root = 0                                    */
    int32_t form;              /* GRTX_FORM_*                                              */
    int32_t sh_degree;
    int32_t reserved;
    int64_t bytes_nodes;       /* device bytes of BVH nodes                                */
    int64_t bytes_leaves;      /* device bytes of leaf records (geometry / triangles, and   */
                               /* the raw parameters in leaf order that the backward reads) */
    int64_t bytes_appearance;  /* device bytes of the appearance (SH) records              */
    int64_t bytes_workspace;   /* device bytes of the per-slot checkpoint/eviction buffers */
    float bounds[6];           /* world AABB of all leaves                                 */
} grtx_scene_info;

typedef struct grtx_scene grtx_scene;

/* ---------------------------------------------------------------------------------------- */
/* Utilities                                                                                */
/* ---------------------------------------------------------------------------------------- */

/* Static English text for a status code (never NULL). */
GRTX_API const char *grtx_status_string(int status);
/* GRTX_VERSION of the library. */
GRTX_API int grtx_version(void);
/* Host-side text of the last error detected in this thread (never NULL; "" if none). */
GRTX_API const char *grtx_last_error(void);

/* The library allocates its device memory (scene arrays, build temporaries, trace
 * workspaces) stream-ordered from a pool of its own on each device, which keeps freed memory
 * mapped for the next build or trace. grtx_memory_trim synchronises the current device and
 * returns the pool's unused memory to the driver beyond keep_bytes (>= 0). Memory of live
 * scenes, worlds and servers is not affected. */
GRTX_API int grtx_memory_trim(int64_t keep_bytes);

/* ---------------------------------------------------------------------------------------- */
/* Building blocks of the BVH build (each also runs inside grtx_build_bvh)                  */
/* ---------------------------------------------------------------------------------------- */

/* Parameter activation and instance transform (Sec. II-B; Sec. IV-A: the per-Gaussian
 * transform, built from its rotation and scales, that takes a ray into unit-sphere space).
 * For each Gaussian i: o = sigmoid(logit); s = exp(log_scale); R from the normalised
 * quaternion; kappa = sqrt(2 ln(o/alpha_min)). If o > alpha_min, writes
 *   d_geom[i] (16 floats): the rows of A = diag(1/(kappa s)) R^T with the mean, as three float4
 *     (A_j0, A_j1, A_j2, mu_j), so that x_unit = A (x - mu); then (o, -0.5 kappa^2 log2(e),
 *     bits of i, 0);
 *   d_aabb[i] (6 floats): lo xyz, hi xyz of the ellipsoid {x : |A x + b| <= 1}, widened by a
 *     relative 4e-6 so it stays conservative under FP32 rounding;
 * otherwise d_geom[i] is all zero and d_aabb[i] is the empty box (+inf, -inf).
 * d_geom, d_aabb: device, caller-owned, 16-byte aligned. */
GRTX_API int grtx_prep_gaussians(const grtx_gaussians *g, float alpha_min, float *d_geom,
                                 float *d_aabb, void *stream);

/* Morton order of AABB centroids (LBVH construction; the paper builds its BVH with a
 * third-party builder, Sec. V-A). centroid = 0.5 (lo + hi) in FP32; each coordinate is
 * quantised to 21 bits as floor((c - blo) * (2^21 / (bhi - blo))) clamped to [0, 2^21 - 1]
 * (0 when bhi == blo), all in FP32, and the bits are interleaved x, y, z from the most
 * significant triple down into a 63-bit code. An empty box (lo > hi on any axis) gets the
 * code 2^64 - 1. d_bounds: device float[6] (lo xyz, hi xyz) of the centroids, or NULL to
 * have them computed over the non-empty boxes (written to d_bounds_out if non-NULL).
 * d_aabb [n][6] in, d_codes [n] out; device, caller-owned. */
GRTX_API int grtx_morton_codes(const float *d_aabb, int64_t n, const float *d_bounds,
                               float *d_bounds_out, uint64_t *d_codes, void *stream);

/* Size-aware 64-bit Morton codes (extended Morton codes, Vinkler, Bittner and Havran, HPG
 * 2017; the paper builds its BVH with a third-party builder, Sec. V-A): the box diagonal is a
 * fourth coordinate, so that Gaussians of very different sizes (scales spanning three
 * decades) do not share subtrees whose boxes the largest of them inflate. In FP32 per box:
 * q_a = floor((c_a - blo_a) * (2^16 / (bhi_a - blo_a))) clamped to [0, 2^16 - 1] for the
 * centroid c = 0.5 (lo + hi) (0 when bhi_a == blo_a); q_s = floor(sqrt((ex^2 + ey^2) + ez^2)
 * * (2^15 / E)) clamped to [0, 2^16 - 2], with e = hi - lo and E the largest extent of the
 * centroid bounds (q_s = 0 when E == 0). Bit b of (q_x, q_y, q_z, q_s) is code bit
 * 4b + (3, 2, 1, 0). An empty box gets 2^64 - 1, which no other code reaches. Arguments
 * and bounds as for grtx_morton_codes. */
GRTX_API int grtx_morton_codes_sized(const float *d_aabb, int64_t n, const float *d_bounds,
                                     float *d_bounds_out, uint64_t *d_codes, void *stream);

/* Stable ascending LSD radix sort of (key, value) pairs in place, over the low key_bits bits
 * of the keys (1..64; bits above are ignored for ordering). d_temp / *temp_bytes: scratch;
 * call with d_temp == NULL to get the required size in *temp_bytes (nothing is enqueued).
 * d_keys [n], d_values [n], d_temp: device, caller-owned. n < 2^31. */
GRTX_API int grtx_sort_pairs(uint64_t *d_keys, uint32_t *d_values, int64_t n, int key_bits,
                             void *d_temp, size_t *temp_bytes, void *stream);

/* Binary radix tree over n >= 2 sorted keys (index appended to break ties between equal
 * keys): internal node 0 is the root; node i covers a key range with i at one end; a range
 * [a, b] split at g has children [a, g] and [g+1, b], numbered g and g+1 if internal or
 * encoded as (0x80000000 | leaf index) if they hold one key. Writes d_left / d_right [n-1]
 * and d_parent [2n-1] (entries 0..n-2: internal nodes, n-1+j: leaf j; root's is 0xFFFFFFFF).
 * Device, caller-owned. */
GRTX_API int grtx_radix_tree(const uint64_t *d_sorted_keys, int64_t n, uint32_t *d_left,
                             uint32_t *d_right, uint32_t *d_parent, void *stream);

/* Locally-ordered clustering (PLOC: Meister and Bittner, IEEE TVCG 2018; the paper builds its
 * BVH with a third-party SAH builder, Sec. V-A) over n >= 2 leaf boxes in Morton order
 * (d_leaf_aabb [n][6]). Iterate until one cluster is left: every cluster i picks the cluster
 * j in [i - GRTX_PLOC_RADIUS, i + GRTX_PLOC_RADIUS] whose union box has the smallest surface
 * area 2 (ex ey + ey ez + ez ex) (FP32, rounded in that order), ties to the lower j; each
 * mutual pair i < j merges into a new node (left = cluster i, right = cluster j) in cluster
 * i's place, new nodes numbered in creation order by increasing i; the clusters are
 * compacted in order. The node created k-th becomes internal node n - 2 - k (the root is 0).
 * Writes d_left / d_right [n-1] and d_parent [2n-1] in grtx_radix_tree's layout and, if not
 * NULL, *iterations (host). Allocates scratch stream-ordered and synchronises the stream
 * once per iteration (to read how many clusters are left). Device, caller-owned. */
GRTX_API int grtx_ploc_tree(const float *d_leaf_aabb, int64_t n, uint32_t *d_left, uint32_t *d_right,
                            uint32_t *d_parent, int *iterations, void *stream);

/* Bottom-up bounds: box of every internal node = union of its children's boxes, leaves'
 * boxes given in sorted order (d_leaf_aabb [n][6]); FP32 min/max, hence exact. Uses the tree
 * of grtx_radix_tree. d_node_aabb [n-1][6] out; d_counters: device scratch of n-1 uint32
 * (contents on entry ignored). Device, caller-owned. */
GRTX_API int grtx_refit(const uint32_t *d_left, const uint32_t *d_right, const uint32_t *d_parent,
                        const float *d_leaf_aabb, int64_t n, float *d_node_aabb,
                        uint32_t *d_counters, void *stream);

/* ---------------------------------------------------------------------------------------- */
/* Scenes                                                                                   */
/* ---------------------------------------------------------------------------------------- */

/* Build the acceleration structure for one set of Gaussians (Sec. IV-A "Bounding
 * Primitives": form GRTX_FORM_SPHERE keeps one instance per Gaussian over a shared analytic
 * unit sphere; GRTX_FORM_ICO20 / GRTX_FORM_ICO80 build the same instance BVH and refer to a
 * shared template mesh BVH (grtx_template_mesh), uploaded once per device; GRTX_FORM_PROXY20
 * is the 20-triangle monolithic baseline of Sec. III-C).
 * Steps: grtx_prep_gaussians -> (proxy: expand 20 triangles per Gaussian) -> Morton codes ->
 * radix sort -> radix tree -> refit -> node compaction. p->alpha_min fixes the ellipsoid
 * radius; later traces must use the same alpha_min. The library allocates (stream-ordered)
 * and owns all scene memory: packed copies of the geometry and appearance, the BVH and a
 * per-slot trace workspace grown on demand; the caller's arrays may be freed once the
 * stream passes the call. Synchronises the stream once at the end (to read the node count
 * and tree depth). *out is set only on success. Fails with GRTX_ERR_OVERFLOW_FATAL if the
 * tree is deeper than the traversal stack (128). */
GRTX_API int grtx_build_bvh(const grtx_gaussians *g, const grtx_params *p, int form, void *stream,
                            grtx_scene **out);

/* Update modes of grtx_scene_update. */
#define GRTX_UPDATE_REFIT 0
#define GRTX_UPDATE_REBUILD 1

/* Update a built scene in place for new parameters of the same Gaussians, as a training loop
 * needs after each optimiser step. g must have the scene's n and sh_degree; the scene keeps its
 * form, alpha_min, Morton code kind and builder.
 * GRTX_UPDATE_REFIT (sphere and icosphere forms) keeps the tree's topology and leaf order. It
 * recomputes every leaf's record, appearance and box from g (Sec. IV-A's per-Gaussian
 * bounds), then refits the node boxes bottom-up, the last step of the LBVH build. A leaf whose
 * Gaussian is now at or below alpha_min gets an empty box and a record that never hits. A
 * Gaussian culled at the last build cannot be added by a refit: if one is now above alpha_min,
 * the scene is rebuilt instead, and *rebuilt (may be NULL) is set to 1.
 * GRTX_UPDATE_REBUILD always runs the full build of grtx_build_bvh (any form) and sets
 * *rebuilt to 1. A refit leaves every array in place; a rebuild replaces them, freeing the old
 * ones stream-ordered on `stream`, and keeps the trace workspace.
 * Images do not depend on which happened: the tree only sets the traversal cost. Earlier work
 * on the scene must be ordered before `stream`, which becomes the scene's stream. A world
 * placing the scene needs grtx_world_update afterwards (its object bounds moved), and a
 * server must not hold a scene while it is rebuilt. Synchronises the stream once (refit: to
 * read the revival flag and the root box).
 * Errors: GRTX_ERR_INVALID_ARG for a NULL scene, bad arrays, another n or sh_degree, an
 * unknown mode, or a refit of the proxy form (the scene is unchanged then); after a CUDA or
 * build error the scene may only be updated again or destroyed. */
GRTX_API int grtx_scene_update(grtx_scene *scene, const grtx_gaussians *g, int mode, void *stream,
                               int *rebuilt);

/* The shared template mesh of GRTX_FORM_ICO20 / GRTX_FORM_ICO80 (host only, no device work):
 * a regular icosahedron (20 triangles), or for ICO80 the icosphere made by splitting each of
 * its faces into four at the edge midpoints pushed out to the sphere, with every face oriented
 * outwards and the mesh scaled so that its nearest face plane is at 1 + 1e-3 from the centre
 * (it encloses the unit sphere). Writes *n_tris and, if h_tris is not NULL, the triangles as
 * h_tris[n_tris][9] (three vertices x, y, z) into caller host memory of 9 * n_tris floats.
 * At a top-level leaf the trace maps the ray into the Gaussian's unit-sphere space (scaled by
 * 1 / (1 + 1e-5 + 4e-6 |o_l|) against FP32 rounding, which leaves t unchanged), traverses a
 * BVH over these triangles, and on a triangle hit at t > t_near runs the exact unit-sphere
 * test for the Gaussian, so the image equals the sphere form's. */
GRTX_API int grtx_template_mesh(int form, float *h_tris, int *n_tris);

/* Fill *info (host) for a built scene. Host-only, no stream work. */
GRTX_API int grtx_scene_info_get(const grtx_scene *scene, grtx_scene_info *info);

/* Copy the scene's internal arrays to caller device buffers (for tests and tools); any
 * pointer may be NULL. d_nodes: [n_nodes][16] floats (child 0 box lo xyz, hi x | hi yz,
 * child 1 box lo xy | lo z, hi xyz | child refs as uint32 bits, then per child the largest
 * proxy diameter in its subtree, 0 for the sphere form); d_leaf_ids: [n_leaves]
 * uint32 Gaussian id of each leaf in leaf order; d_codes: [n_leaves] sorted Morton codes. */
GRTX_API int grtx_scene_export(const grtx_scene *scene, float *d_nodes, uint32_t *d_leaf_ids,
                               uint64_t *d_codes, void *stream);

/* Release a scene (stream-ordered on the scene's build stream; NULL is a no-op). */
GRTX_API void grtx_scene_destroy(grtx_scene *scene);

/* ---------------------------------------------------------------------------------------- */
/* Rendering                                                                                */
/* ---------------------------------------------------------------------------------------- */

/* The rays a camera generates (for tests; the trace kernels generate them in-kernel).
 * d_origins / d_dirs [n][3], d_tnear / d_tfar [n]; device, caller-owned; n = W*H. */
GRTX_API int grtx_generate_rays(const grtx_camera *cam, float *d_origins, float *d_dirs,
                                float *d_tnear, float *d_tfar, void *stream);

/* Render every ray of cam (Sec. III-A pipeline: ray generation, traversal gathering the k
 * nearest hits per round, blending in depth order, early termination; Sec. IV-B checkpointed
 * resume). Hits are Gaussians whose max response along the ray (Sec. III-A Eq. t-max-resp)
 * reaches alpha_min with t_near < t_alpha <= t_far, ordered by (t_alpha, leaf index); colour
 * is max(0, SH(ray direction) + 0.5). One persistent launch; per resident ray slot the
 * checkpoint lists and eviction list live in the scene's workspace (grown on demand with a
 * stream-ordered allocation). */
GRTX_API int grtx_trace_forward(grtx_scene *scene, const grtx_camera *cam, const grtx_params *p,
                                const grtx_trace_outputs *out, void *stream);

#define GRTX_MAX_BATCH 64

/* Trace several cameras or ray lists of one scene in one persistent launch (the segments of
 * the serving kernel): cams[i] is traced into rgbT[i] (device [width*height][4], 16-byte
 * aligned, as grtx_trace_forward's rgbT), with the same parameters for all. The warps of
 * every item share the GPU, so a small list (a frame's bounce rays) overlaps a large image
 * instead of running after it with most of the GPU idle. The launch's queue hands out the
 * views smallest first, whatever their order in cams, so that a small view of long rays runs
 * beside the large ones rather than after them. Results equal grtx_trace_forward's
 * for each camera alone, to the last bit of rounding (the batch runs in the serving kernel).
 * Sphere-form scenes, checkpoint or restart traversal, no optional outputs; n_cams in
 * [1, GRTX_MAX_BATCH].
 * Errors: GRTX_ERR_INVALID_ARG for bad arguments (checked before any device work). */
GRTX_API int grtx_trace_forward_batch(grtx_scene *scene, const grtx_camera *cams, int n_cams,
                                      const grtx_params *p, float *const *rgbT, void *stream);

/* Gradients of a loss L w.r.t. the raw Gaussian parameters for the image of
 * grtx_trace_forward. g must hold the parameters the scene was built from; d_rgbT is the
 * forward output [n_rays][4] and d_dL_drgbT the upstream gradient [n_rays][4]. The kernel
 * re-traverses the same rounds and accumulates, front to back, the derivative of Eq.
 * volume-render and of alpha = o G(r_o + t_alpha r_d) through the unit-sphere transform
 * (the hit set, order and termination index are piecewise constant and not differentiated).
 * Accumulates into *grads (caller zeroes): SH gradients with vector atomics, the others with
 * vector atomics into a per-leaf stage that a second kernel adds into *grads. The gradient
 * reads the scene's own copy of the raw parameters (packed in leaf order at build and
 * update), so g must be the parameters the scene was built or last updated from. */
GRTX_API int grtx_trace_backward(grtx_scene *scene, const grtx_gaussians *g,
                                 const grtx_camera *cam, const grtx_params *p,
                                 const float *d_rgbT, const float *d_dL_drgbT,
                                 const grtx_grads *grads, void *stream);

/* grtx_trace_backward for a forward that saved its blend lists (grtx_trace_outputs.saved,
 * same scene, camera and parameters): a ray with a complete list (n <= cap) computes its
 * gradients from the list, in blend order, without traversing the BVH; the others replay
 * their rounds as in grtx_trace_backward. The gradients are the same (up to the order of the
 * atomic additions). Sphere form. */
GRTX_API int grtx_trace_backward_saved(grtx_scene *scene, const grtx_gaussians *g,
                                       const grtx_camera *cam, const grtx_params *p,
                                       const float *d_rgbT, const float *d_dL_drgbT,
                                       const grtx_saved *saved, const grtx_grads *grads,
                                       void *stream);

/* A rectangular planar mirror for secondary rays (Sec. VI "GRTX-HW on Secondary Rays").
 * center: a point of the mirror; normal: unit normal; axis_u / axis_v: unit in-plane axes;
 * the mirror is {center + a axis_u + b axis_v : |a| <= half_u, |b| <= half_v}.
 * t_near_secondary: t_near of the reflected rays (keeps them off the mirror). */
typedef struct grtx_mirror {
    float center[3], normal[3], axis_u[3], axis_v[3];
    float half_u, half_v;
    float t_near_secondary;
    float reserved;
} grtx_mirror;

/* Rays of a camera with one mirror bounce. Every primary ray (width*height, pixel order) is
 * written to the d_prim_* arrays with t_far clipped to the mirror where it hits it (in
 * (t_near, t_far)). Each primary that hits spawns one secondary ray: origin at the hit point,
 * direction reflected about the normal (d - 2 (d.n) n), t_near = m->t_near_secondary,
 * t_far = +inf. Secondaries are compacted into d_sec_* (capacity width*height) with their
 * pixel in d_sec_pixel; their count is written to *d_n_sec (device). The order of the
 * secondary list is unspecified; d_sec_pixel identifies each ray. All device, caller-owned:
 * origins/dirs [n][3], tnear/tfar [n]. */
GRTX_API int grtx_mirror_rays(const grtx_camera *cam, const grtx_mirror *m, float *d_prim_origins,
                              float *d_prim_dirs, float *d_prim_tnear, float *d_prim_tfar,
                              float *d_sec_origins, float *d_sec_dirs, float *d_sec_tnear,
                              float *d_sec_tfar, int32_t *d_sec_pixel, int32_t *d_n_sec,
                              void *stream);

/* A solid glass ball for refraction secondary rays (Sec. VI "GRTX-HW on Secondary Rays": a
 * spherical glass object placed in the scene). center, radius > 0; ior: index of refraction
 * (> 0) against the surrounding air of index 1; t_near_secondary: t_near of its rays. */
typedef struct grtx_glass {
    float center[3];
    float radius;
    float ior;
    float t_near_secondary;
    float reserved[2];
} grtx_glass;

#define GRTX_MAX_BOUNCE_OBJECTS 16

/* Rays of a camera with one bounce off the nearest of n_mirrors mirrors and n_glass glass
 * balls (host arrays, each count in [0, GRTX_MAX_BOUNCE_OBJECTS], copied at the call). Every
 * primary ray (width*height, pixel order) is written to d_prim_* with t_far clipped to the
 * nearest object it meets in (t_near, t_far). Each such primary spawns one secondary ray with
 * t_near = the object's t_near_secondary and t_far = +inf:
 *  - mirror: as grtx_mirror_rays (origin at the hit, direction reflected about the normal);
 *  - glass: the unit direction is refracted into the ball at the entry point (Snell's law,
 *    index 1 outside), carried straight across the ball to the far side, and refracted out;
 *    the secondary starts on the far side with that unit direction. The inside of a ball is
 *    empty (nothing is rendered along the chord), there is no Fresnel reflection, and a ray
 *    that starts inside a ball or only grazes it does not meet it.
 * Output layout, compaction and *d_n_sec as for grtx_mirror_rays. */
GRTX_API int grtx_secondary_rays(const grtx_camera *cam, const grtx_mirror *mirrors, int n_mirrors,
                                 const grtx_glass *glass, int n_glass, float *d_prim_origins,
                                 float *d_prim_dirs, float *d_prim_tnear, float *d_prim_tfar,
                                 float *d_sec_origins, float *d_sec_dirs, float *d_sec_tnear,
                                 float *d_sec_tfar, int32_t *d_sec_pixel, int32_t *d_n_sec,
                                 void *stream);

/* Composite the secondary image behind the primary one: for each of the *d_n_sec secondary
 * rays j (at most max_sec) with pixel p = d_sec_pixel[j], the primary pixel (C + T bg, T)
 * becomes (C + T C2, T T2) where (C2, T2) = d_sec_rgbT[j] rendered with the same bg, i.e.
 * the reflection replaces the primary's background term (Eq. volume-render continued past
 * the mirror). d_rgbT [n_pixels][4] in/out, d_sec_rgbT [max_sec][4]; device, 16-byte aligned. */
GRTX_API int grtx_composite_bounce(float *d_rgbT, const float *d_sec_rgbT, const int32_t *d_sec_pixel,
                                   const int32_t *d_n_sec, int64_t max_sec, const float bg[3],
                                   void *stream);

/* ---------------------------------------------------------------------------------------- */
/* Allocation-free forward trace                                                             */
/* ---------------------------------------------------------------------------------------- */

/* The paper has no counterpart to this entry point. It is for callers that must not allocate
 * device memory while they render: a renderer that reserves its whole memory budget at
 * start-up and may not grow it, or a frame loop that cannot afford to wait on the allocator.
 * grtx_trace_forward may allocate (it grows a per-scene workspace on first use); this variant
 * never does. It renders cam like grtx_trace_forward with rgbT = d_rgbT (device [n_rays][4],
 * 16-byte aligned, caller-owned) and no optional outputs; GRTX_TRAVERSAL_SINGLE is rejected
 * with GRTX_ERR_INVALID_ARG (its hit lists do not fit the array). Its scratch -- the ray-queue
 * counter and the per-ray-slot checkpoint and eviction lists -- lives in one library-owned
 * device array of GRTX_NOALLOC_SCRATCH_BYTES (32 MiB) that every GPU which loads the library
 * holds until the process exits. The number of rays in flight is whatever fits in that array:
 * floor((GRTX_NOALLOC_SCRATCH_BYTES - 256) / (128 * (2 C + E) * 8)) blocks of 128 ray slots
 * (C, E the checkpoint and eviction capacities; C = E = 1 for restart traversal), at most the
 * resident blocks of the GPU. With the default capacities 256 / 512 that is 31 blocks, 3,968
 * rays, against 155,648 for grtx_trace_forward at k = 16 on 152 SMs, so a frame may take
 * longer; restart traversal fills the GPU. If one block of 128 ray slots
 * does not fit (large ckpt_capacity / evict_capacity) it returns GRTX_ERR_INVALID_ARG and says
 * so in grtx_last_error(). The first call on a device looks up the array's device address
 * with that device current; make that first call before any stream capture begins. Every
 * call uses the same array: calls whose work overlaps on the GPU (different streams, or
 * threads without ordering) race and produce wrong images, so order them on one stream. */
#define GRTX_NOALLOC_SCRATCH_BYTES (32u << 20)
GRTX_API int grtx_trace_forward_noalloc(grtx_scene *scene, const grtx_camera *cam,
                                        const grtx_params *p, float *d_rgbT, void *stream);

/* ---------------------------------------------------------------------------------------- */
/* Multi-level instancing (Sec. VI "Support for Dynamic and Multi-Object Scenes"): a shared  */
/* primitive (the unit sphere), per-object instance BVHs (built scenes), a scene-level TLAS. */
/* ---------------------------------------------------------------------------------------- */

/* One placement of a built sphere-form scene: x_world = L x_object + c with object_to_world
 * = rows (L_r0 | c_0), (L_r1 | c_1), (L_r2 | c_2) (row-major 3x4, L invertible). The scene
 * is not owned and must outlive every world that refers to it; one scene may be placed many
 * times. */
typedef struct grtx_instance {
    const grtx_scene *scene;
    float object_to_world[12];
    int32_t reserved[2];
} grtx_instance;

typedef struct grtx_world grtx_world;

/* Build a world over n >= 1 instances (host array, copied). All scenes must be of
 * GRTX_FORM_SPHERE and built with the same alpha_min. The host computes each instance's
 * world-to-object map (in double, stored as FP32) and world box (the object's bounds through
 * the map, widened by 1e-5 of its extent + 1e-6 of its coordinates against FP32 rounding)
 * and builds the scene-level BVH over the boxes of the non-empty instances; the instance
 * table and the TLAS go to device memory on `stream`. World Gaussian ids: the instance's
 * base (the sum of the n of the scenes of the instances before it) plus the Gaussian's id
 * in its scene. Fails with GRTX_ERR_INVALID_ARG on a NULL or non-sphere scene, mixed
 * alpha_min, a non-invertible or non-finite map, more than 2^32 - 2 leaves in all, or a
 * TLAS deeper than 32. */
GRTX_API int grtx_world_create(const grtx_instance *inst, int n, void *stream, grtx_world **out);

/* Replace the instance list (objects moved, added or removed): rebuilds the TLAS and the
 * instance table, as grtx_world_create. Waits for the world's earlier work on `stream`. */
GRTX_API int grtx_world_update(grtx_world *world, const grtx_instance *inst, int n, void *stream);

/* Render cam through the world: k-buffer rounds (k = 8, 16 or 32) with checkpointed resume
 * or restart (GRTX_TRAVERSAL_CHECKPOINT / RESTART) over the two-level structure. At a TLAS
 * leaf the ray is mapped into the object's frame (t is unchanged by the affine map) and
 * descends that scene's BVH; checkpoint entries carry the instance of object-level nodes
 * (Sec. IV-B's checkpoint entry with its TLAS-leaf field). Keys are (t, world leaf index)
 * and colours are evaluated along the object-frame direction. Outputs as
 * grtx_trace_forward, with blended_ids in world Gaussian ids. p->alpha_min must be the
 * scenes'. The world's trace workspace is grown on demand (stream-ordered allocation). */
GRTX_API int grtx_world_trace_forward(grtx_world *world, const grtx_camera *cam, const grtx_params *p,
                                      const grtx_trace_outputs *out, void *stream);

/* Release a world (waits for its work on the last stream it used; NULL is a no-op). */
GRTX_API void grtx_world_destroy(grtx_world *world);

/* ---------------------------------------------------------------------------------------- */
/* Serving: several resident scenes, camera requests batched into persistent launches.      */
/* ---------------------------------------------------------------------------------------- */

typedef struct grtx_server grtx_server;

/* A camera request: render cam on scene scene_id into d_rgbT (device [W*H][4], 16-byte
 * aligned, caller-owned, valid until the request completes), or, with d_rgbT = NULL, into an
 * output the server allocates from its memory budget when it admits the request (see
 * grtx_server_create; returned in the completion, given back with grtx_server_release).
 * tag is returned with the completion. */
typedef struct grtx_request {
    int32_t scene_id;
    int32_t reserved;
    grtx_camera cam;
    float *d_rgbT;
    uint64_t tag;
} grtx_request;

/* A finished request: tag, status, host wall-clock times in seconds (CLOCK_MONOTONIC) of
 * admission and completion (the host saw its last tile written), and the device image
 * [W*H][4] it was rendered into (the request's own buffer or a server-owned one). */
typedef struct grtx_completion {
    uint64_t tag;
    int32_t status;
    int32_t reserved;
    double t_admit;
    double t_done;
    float *d_rgbT;
} grtx_completion;

/* Create a server over n_scenes built scenes (not owned; they must outlive the server).
 * p: tracing parameters for every request (checkpoint or restart traversal;
 * GRTX_TRAVERSAL_SINGLE is rejected with GRTX_ERR_INVALID_ARG). Host call; waits for the
 * device once (the scenes' builds). A request's output is complete when its completion is
 * reported.
 *
 * Scheduling. A step is one persistent launch of the server's trace kernel; its queue hands
 * out 32-ray tiles of the admitted requests (mixed scenes and resolutions). The running
 * ("live") launch is fed while it runs: the host publishes up to max_rays_per_step more rays
 * (0: two rounds of the launch's warps, 32 rays each: 311,296 at full residency on 152 SMs)
 * whenever less than half of that is left unclaimed, choosing the requests by deadline (see
 * grtx_server_set_order), so that a request that arrives waits for at most about that much
 * of others' work. Warps without work wait for more (see grtx_server_set_linger). A launch's
 * segment table holds 4 x max_inflight pieces of requests; when it is full, or the launch has
 * gone idle, the next work starts a new launch in a free step slot while the old one
 * finishes. max_inflight: requests admitted at once (0: 64).
 *
 * Memory (the paper sizes its checkpoint and eviction buffers per resident ray slot and
 * reports their total, Sec. V-E). The server runs up to 2 step slots, each with its own
 * stream (slot 0 uses `stream`, the other a stream the server creates), queue counter and
 * checkpoint/eviction lists, so that a new launch fills the SMs the finishing launch's last
 * warps leave (a third slot gave the same latency and throughput; a single slot makes each
 * new launch wait for the previous one to end). One step slot's lists take (resident ray
 * slots) x (2 ckpt_capacity + evict_capacity) x 8 bytes: 1.27 GB with the default
 * capacities at full residency on 152 SMs.
 *   - mem_budget_bytes = 0: no cap. 2 step slots at full residency; requests must bring their
 *     own output (d_rgbT = NULL is rejected with GRTX_ERR_INVALID_ARG).
 *   - mem_budget_bytes > 0: the server's device memory never exceeds it. The step slots' lists
 *     take at most half of it: as many full-residency step slots as fit (1 or 2), or one slot
 *     with as many 128-ray blocks as fit; GRTX_ERR_INVALID_ARG if not even one block of lists
 *     fits. The rest (less the small segment tables) is reserved as an output arena. A request
 *     with d_rgbT = NULL needs W*H*16 bytes of it: requests are admitted in submission order,
 *     and admission stops at the first one whose output does not fit until grtx_server_release
 *     returns memory (so a large request is never overtaken). A request whose output exceeds
 *     the whole arena is rejected by grtx_server_submit with GRTX_ERR_OOM.
 * An allocation that fails returns GRTX_ERR_OOM. */
GRTX_API int grtx_server_create(grtx_scene *const *scenes, int n_scenes, const grtx_params *p,
                                int64_t mem_budget_bytes, int64_t max_rays_per_step, int max_inflight,
                                void *stream, grtx_server **out);

/* Give a server-owned output (a completion's d_rgbT of a request submitted with d_rgbT =
 * NULL) back to the server's arena. Call it once every read of the image has completed
 * (the server may render the next admitted request into the same memory). Host call.
 * GRTX_ERR_NOT_FOUND if d_rgbT is not a live server-owned output. */
GRTX_API int grtx_server_release(grtx_server *srv, float *d_rgbT);

/* How long, in nanoseconds, a running step launch that has run out of work stays open for
 * more while admitted requests are still in flight (default 2,000,000: 2 ms). Work that
 * arrives while a launch is open is appended to it (its warps take it without a new launch);
 * the host closes the launch (its waiting warps stop) when no admitted request is left, when it
 * has had no work for linger_ns (checked by grtx_server_poll), or when its segment table is
 * full. As a backstop for a caller that stops polling, waiting warps stop on their own after
 * 16 x linger_ns without a publication (at least 20 ms, at most 1 s); a tile published to a
 * warp that has stopped is traced by a later launch. Waiting warps keep their SMs: kernels of
 * other streams start on them once the launch ends. 0: a launch ends as soon as its published
 * work is taken (its warps do not wait). Applies to launches started after the call. Host
 * call. GRTX_ERR_INVALID_ARG if linger_ns is negative or above 1 s. */
GRTX_API int grtx_server_set_linger(grtx_server *srv, int64_t linger_ns);

/* on = 1 (the default): waiting warps stop on their own only after the backstop described at
 * grtx_server_set_linger, so that appends do not race with warps giving up. on = 0: they stop
 * linger_ns after the last publication, and the host appends to any launch none of whose warps
 * it has seen stop, so that appends race with warps giving up; tiles published to warps that
 * have stopped are then traced by a later launch (the recovery every launch has, exercised
 * often). Same images either way. Applies to launches started after the call. Host call. */
GRTX_API int grtx_server_set_append_guard(grtx_server *srv, int on);

/* Order in which admitted requests' work is published to the running launch: by deadline,
 * admission time + size_ns_per_ray x the request's rays (default 5 ns per ray). 0: admission
 * order; large: the smallest request first. Host call. GRTX_ERR_INVALID_ARG unless
 * 0 <= size_ns_per_ray <= 1e9. */
GRTX_API int grtx_server_set_order(grtx_server *srv, double size_ns_per_ray);

/* Sizes chosen at creation and current use (host call). */
typedef struct grtx_server_info {
    int32_t n_step_slots;        /* step slots (streams) the server runs, 1 or 2           */
    int32_t blocks_per_step;     /* 128-ray blocks of one step's persistent launch          */
    int64_t list_bytes;          /* checkpoint/eviction lists of all step slots             */
    int64_t arena_bytes;         /* output arena reserved for server-owned outputs          */
    int64_t arena_used;          /* bytes of the arena held by admitted, unreleased outputs */
    int64_t device_bytes;        /* all device memory the server holds                      */
    int32_t n_inflight;          /* admitted, not yet returned by grtx_server_poll           */
    int32_t n_pending;           /* submitted, not yet admitted                            */
    int64_t n_launches;          /* step launches so far                                    */
    int64_t n_appends;           /* publications of new work to a running launch so far     */
    int64_t n_retried_tiles;     /* 32-ray tiles a launch gave up and a later one traced    */
} grtx_server_info;
GRTX_API int grtx_server_get_info(const grtx_server *srv, grtx_server_info *info);

/* Queue n requests (host array, copied). Non-blocking. None of them is queued if one fails:
 * GRTX_ERR_BUSY if the pending queue would exceed 65536 entries; GRTX_ERR_OOM for a request
 * with d_rgbT = NULL whose output exceeds the server's whole output arena (or with no budget,
 * GRTX_ERR_INVALID_ARG); GRTX_ERR_NOT_FOUND for an unknown scene id. */
GRTX_API int grtx_server_submit(grtx_server *srv, const grtx_request *reqs, int n);

/* Take completed requests. The server's scheduler thread (started by grtx_server_create, ended
 * by grtx_server_destroy) does the rest on its own, every 20 us while there is work: it admits
 * pending requests (continuous batching), publishes work to the live launch or starts a launch
 * (see grtx_server_create), and completes requests whose tiles have all been traced (each piece
 * of a request raises a flag in host memory when its last tile is written). Writes at most
 * max_done completions to done (host) and their count to *n_done. Non-blocking unless
 * wait != 0, in which case it blocks until at least one request has completed or none is
 * admitted. A failure of the scheduler thread (a CUDA error) is returned by every poll from
 * then on. The server's calls may come from any host thread. */
GRTX_API int grtx_server_poll(grtx_server *srv, grtx_completion *done, int max_done, int *n_done,
                              int wait);

/* Submit n requests and poll until all of them complete (a blocking convenience over
 * grtx_server_submit / grtx_server_poll). done: host array of n completions. */
GRTX_API int grtx_render_requests(grtx_server *srv, const grtx_request *reqs, int n,
                                  grtx_completion *done, int *n_done, void *stream);

/* Number of requests admitted but not yet returned by grtx_server_poll, and pending in the
 * queue. */
GRTX_API int grtx_server_load(const grtx_server *srv, int *n_inflight, int *n_pending);

/* Stop the scheduler thread, close the running launches (their waiting warps stop), wait for
 * all in-flight work and release the server (NULL is a no-op). */
GRTX_API void grtx_server_destroy(grtx_server *srv);

#ifdef __cplusplus
}
#endif

#endif /* GRTX_H */
