/*
 * capt.h - C ABI of the GB300 collision-affording point tree (CAPT) library.
 *
 * The CAPT (Ramsey, Kingston, Thomason, Kavraki, 2024) answers "does a sphere of
 * radius r in [r_min, r_max] centred at x touch any point of a cloud?" exactly
 * (Lemma 1, Sec. V-B) with a fixed-length descent of an Eytzinger-ordered split
 * sequence T to a leaf cell (Alg. 3, Sec. IV-D), a test against that leaf's
 * bounding box A_i, and a scan of the leaf's affordance set P_i.
 *
 * Conventions for every entry point:
 *  - Every call returns a capt_status (0 = CAPT_OK, negative = error) and never throws.
 *    capt_last_error() gives a message for the calling thread's last error.
 *  - "host" pointers are CPU memory; "device" pointers are CUDA device memory on the
 *    device the tree was uploaded to (for example a torch tensor's data_ptr()).
 *  - Inputs are caller-owned and never retained after the call returns (for device
 *    inputs: after the work queued on the stream has finished).  Outputs go to
 *    caller-owned buffers.  The tree owns its own copies of everything.
 *  - Device calls are asynchronous and stream-ordered on `stream` (a cudaStream_t; NULL
 *    is the legacy default stream).  Errors found while queueing are returned; errors
 *    found by a kernel (a bounded wait that gave up) are latched in the tree's device
 *    status word, read by capt_device_status().
 *  - The sphere, configuration and joint-angle queries hand tiles to their warps from a
 *    work counter of the tree (one of 64, zeroed on `stream` before the launch, once
 *    the launch that last used it has finished, through an event the library records).
 *    Queries on one tree may therefore run on several streams and host threads at
 *    once.  Inside a stream capture they use a fixed tile order instead, so a captured
 *    graph holds no hidden state and replays exactly.
 *  - Queries assume r_min <= r <= r_max (Lemma 1's hypothesis).  Outside that range
 *    the flag is unspecified (it is still computed, never faults).  Non-finite
 *    centres give unspecified flags and never fault.
 *  - All floating-point work on the query path is FP32 with every operation rounded
 *    separately (no fused multiply-add): the flag of a sphere is exactly the FP32
 *    brute-force predicate ((x0-p0)^2 + (x1-p1)^2) + (x2-p2)^2 <= fl(r*r).
 */
#ifndef CAPT_H
#define CAPT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum capt_status {
    CAPT_OK = 0,
    CAPT_E_ARG = -1,        /* null pointer, bad size or bad enum value */
    CAPT_E_RANGE = -2,      /* r_min > r_max, negative or non-finite radius bound */
    CAPT_E_NONFINITE = -3,  /* NaN or infinity in an input point cloud */
    CAPT_E_NOMEM = -4,      /* host or device allocation failed */
    CAPT_E_CUDA = -5,       /* a CUDA runtime call failed (see capt_last_error) */
    CAPT_E_TIMEOUT = -6,    /* a bounded device wait gave up (from capt_device_status) */
    CAPT_E_BOUNDS = -7,     /* a device-side index or size check failed (from capt_device_status) */
    CAPT_E_STATE = -8       /* tree not uploaded, used on another device, or pruned
                               tree given to the clearance calls */
} capt_status;

/* Opaque tree: host arrays plus, after capt_upload, its device layout. */
typedef struct capt_tree capt_tree;

typedef struct capt_tree_stats {
    uint64_t n_points;        /* real points n */
    uint64_t n_leaves;        /* N = 2^L >= max(n, 1), pads at +inf fill N - n leaves */
    uint32_t depth;           /* L, the fixed descent length */
    uint32_t max_set;         /* largest affordance set |P_i| */
    uint64_t total_afforded;  /* sum over leaves of |P_i| */
    uint64_t total_blocks;    /* 4-point blocks in the device point buffer */
    uint64_t pruned_leaves;   /* leaves that kept {t} only (r_min condition, Alg. 1) */
    uint64_t empty_leaves;    /* leaves with |P_i| = 0 */
    uint64_t device_bytes;    /* bytes of the device layout (0 before upload) */
    double build_ms;          /* wall time of capt_build / capt_build_device */
    float r_min, r_max;
    int32_t device;           /* CUDA ordinal after upload, else -1 */
    int32_t build_threads;    /* host threads of capt_build; 0 for capt_build_device */
    uint64_t compact_chunks;  /* capt_compact: 32-point chunks of the Z-ordered cloud (0 before) */
    uint64_t compact_entries; /* capt_compact: sum over leaves of the chunks each lists */
    uint64_t compact_bytes;   /* capt_compact: device bytes of the compact form */
    int32_t full_dropped;     /* 1 if capt_compact freed the replicated device sets */
    int32_t reserved;
    uint64_t scratch_bytes;   /* device scratch the tree allocated on demand (edge work items
                                 of capt_validate_edges, buffers of capt_query_configs_host);
                                 not part of device_bytes */
    uint32_t grid_dims[3];    /* cells per axis of the distance-bound grid (0: none) */
    float grid_cell;          /* its cell side (0: none) */
    uint64_t near_entries;    /* capt_build_near_lists: list entries, padding included (0: none) */
    uint64_t near_bytes;      /* their device bytes (cell table, entries, float4 cloud) */
    uint64_t near_fallback_cells; /* cells whose centres take the paper's path instead */
} capt_tree_stats;

/* ---------------------------------------------------------------------------------
 * Host side (no GPU needed)
 * --------------------------------------------------------------------------------- */

/* Build a CAPT from n points (Alg. 1, Sec. IV-A/B).
 * points: host float[n][3] (x, y, z), copied.  n = 0 is allowed (every query misses).
 * r_min, r_max: the query radius range; 0 <= r_min <= r_max, both finite.  r_min > 0
 *   enables the prune of Alg. 1 (a leaf whose whole cell is within r_min of its
 *   representative stores that point only); r_min = 0 disables it, which the clearance
 *   calls require.
 * Splits cycle x, y, z; each split is the median by (coordinate, point index); a
 * point is afforded by a cell iff its FP64 distance to the closed cell is at most
 * r_max (1 + 1e-5); sets are stored in ascending point index.
 * Errors: CAPT_E_ARG (out == NULL, points == NULL with n > 0, n >= 2^31),
 *         CAPT_E_RANGE, CAPT_E_NONFINITE, CAPT_E_NOMEM. */
int capt_build(const float* points, size_t n, float r_min, float r_max, capt_tree** out);

/* capt_build with an explicit number of host threads (0 = hardware concurrency,
 * 1 = single-threaded).  The result does not depend on the thread count. */
int capt_build_threads(const float* points, size_t n, float r_min, float r_max, int n_threads,
                       capt_tree** out);

/* Space-filling-curve filter (Alg. 2, Sec. IV-C).  For each of the 6 axis
 * permutations (xyz, xzy, yxz, yzx, zxy, zyx) the surviving points are ordered along
 * a Z-order curve (21 bits per axis over the input's bounding box, the permutation's
 * first axis most significant, ties by point index) and a point is kept iff its FP32
 * squared distance to the last kept point exceeds fl(min_spacing^2).
 * points: host float[n][3]; kept_idx: host uint32[n] (caller-owned) receives the kept
 * indices in the last pass's curve order; *n_out their count.
 * Errors: CAPT_E_ARG, CAPT_E_RANGE (min_spacing < 0 or NaN), CAPT_E_NONFINITE, CAPT_E_NOMEM. */
int sfc_filter(const float* points, size_t n, float min_spacing, uint32_t* kept_idx, size_t* n_out);

/* Order of the points along a Z-order curve (the locality measure of Sec. IV-C): 21
 * bits per axis over the input's bounding box, x most significant in every bit triple,
 * ties by point index.  points: host float[n][3]; order: host uint32[n] (caller-owned)
 * receives the permutation.  A cloud relabelled in this order (points[order]) gives a
 * tree whose affordance sets, stored in ascending index, run along the curve, so their
 * 32-point chunks are spatially tight and the chunked scan skips most of them; the
 * filter's output already has this property.  The flags of any query do not depend on
 * the order.  Errors: CAPT_E_ARG, CAPT_E_NONFINITE, CAPT_E_NOMEM. */
int capt_morton_order(const float* points, size_t n, uint32_t* order);

/* sfc_filter on the GPU (Alg. 2, Sec. IV-C): the same kept indices in the same order.
 * Each pass sorts the survivors by Morton key with a stable device radix sort and
 * replaces the sequential sweep by its chain form (the next kept point after p_j is the
 * first later point farther than min_spacing from p_j), marked by pointer doubling.
 * d_points: device float[n][3] on the current device; d_kept: device uint32[n]
 * (caller-owned) receives the kept indices in the last pass's curve order; *n_out
 * (host) their count.  Work is stream-ordered on `stream` and the call synchronises it
 * once (for the count).  The launch sequence of a call depends on n and min_spacing
 * only: the first call for a (device, n, min_spacing) captures it into a CUDA graph
 * with its own buffers (about 90 bytes per point), and later calls of the same size
 * (frame after frame) replay it.  The library keeps the four most recently used such
 * plans until the process exits; calls from several host threads are serialised.
 * Make the first call of a size outside any stream capture of the caller's.  The sweep
 * costs the lengths of the runs of points within min_spacing of each other along the
 * curve (quadratic in a run of coincident points).  On an error the contents of d_kept
 * are unspecified.
 * Errors: CAPT_E_ARG (NULL pointer, n >= 2^31), CAPT_E_RANGE (min_spacing < 0 or NaN),
 *         CAPT_E_NONFINITE, CAPT_E_NOMEM, CAPT_E_CUDA. */
int sfc_filter_device(const float* d_points, size_t n, float min_spacing, uint32_t* d_kept, size_t* n_out,
                      void* stream);

/* Statistics of a tree (host memory).  Errors: CAPT_E_ARG. */
int capt_stats(const capt_tree* t, capt_tree_stats* out);

/* Copy the host arrays of the tree (any output may be NULL):
 * T: float[N-1] split values in Eytzinger order; set_begin: uint64[N+1] offsets;
 * set_idx: uint32[total_afforded] point indices; aabb: float[N][6] (lo xyz, hi xyz;
 * +inf/-inf for an empty set).  Errors: CAPT_E_ARG. */
int capt_export(const capt_tree* t, float* T, uint64_t* set_begin, uint32_t* set_idx, float* aabb);

/* Free host and device memory of the tree and any plan-independent scratch.  NULL-safe.
 * The caller must make sure no queued work still uses the tree. */
void capt_free(capt_tree* t);

/* Message for the last non-OK status returned on the calling thread ("" if none). */
const char* capt_last_error(void);

/* ---------------------------------------------------------------------------------
 * Device side
 * --------------------------------------------------------------------------------- */

/* Copy the tree to device `device` (stream-ordered on `stream`; the host arrays stay).
 * Device layout (all 256-byte aligned):
 *   T      float[N-1 rounded up to 4]  split values (Eytzinger)
 *   leaves 32-byte records {lo.xyz, first block, hi.xyz, count} per leaf
 *   blocks float4[3 * total_blocks]: each set starts at a block of 4 points; the
 *          blocks are stored as three planes, all x quads {x0..x3}, then all y quads,
 *          then all z quads; unused slots hold +inf
 *   ids    uint32[4 * total_blocks] point index per slot (0xffffffff in unused slots)
 *   cloud  float[n][3] the input points (for the clearance gradient)
 *   cbox   float[ceil(total_blocks / 8)][8]: per chunk of 8 consecutive blocks the
 *          FP32 min / max of its finite coordinates {lo.xyz, 0, hi.xyz, 0}; the scan
 *          skips a chunk whose box the sphere does not reach (exact: a box holding p
 *          is never farther than p)
 * Calling it again re-uploads (and releases any compact form of capt_compact).
 * Errors: CAPT_E_ARG, CAPT_E_CUDA, CAPT_E_NOMEM. */
int capt_upload(capt_tree* t, int device, void* stream);

/* Distance-bound grid (this library's addition; the paper has no counterpart): a
 * uniform grid of cubic cells over the cloud's bounding box grown by r_max, at most
 * max_cells cells (0: 2^22), two bytes per cell: a lower and an upper bound of the
 * distance from the cell to the cloud, computed on the device through the tree's own
 * sets (for a point m of each cell, the nearest point of m's leaf set is the nearest
 * cloud point whenever it is within r_max, Lemma 1) and rounded toward the safe side.
 * Configuration queries launched with capt_launch_cfg.grid = 1 classify every sphere
 * that reaches the cloud's bounding box by its cell before any descent: a sphere whose
 * cell is farther than r from the cloud cannot hit, one whose cell is within r of it
 * certainly hits (its configuration is decided at once), only the rest descend.  Both
 * decisions reproduce the FP32 test exactly (the margins are derived in dist_grid.cu),
 * so the flags do not change.  Needs the replicated sets (before capt_compact drops
 * them); a grid built earlier stays valid after the drop.  Rebuilding replaces the old
 * grid; do not call it while queries of this tree run on other streams.  Synchronises
 * `stream`.  Errors: CAPT_E_ARG (max_cells > 2^28), CAPT_E_STATE, CAPT_E_NOMEM,
 * CAPT_E_CUDA. */
int capt_build_grid(capt_tree* t, uint64_t max_cells, void* stream);

/* The distance-bound grid, for tests and inspection.  *info receives its shape (all
 * zero when the tree has none); when h_cells is not NULL it receives the 2 x cells
 * bytes (host buffer, caller-owned): cell (i, j, k) = [origin + (i, j, k) cell,
 * origin + (i + 1, j + 1, k + 1) cell] at index (k dims[1] + j) dims[0] + i holds
 * {lower bound, upper bound} of the distance from the cell (grown by cell / 100 on every
 * side) to the cloud, in units of `unit` (upper bound 255: none).  The kernels locate a
 * centre x by floor(fl(fl(x - origin) * inv_cell)) clamped to the grid.  Synchronous.
 * Errors: CAPT_E_ARG, CAPT_E_CUDA. */
typedef struct capt_grid_info {
    float origin[3];
    float cell;
    float inv_cell;
    float unit;
    int32_t dims[3];
    uint32_t cells;
} capt_grid_info;
int capt_grid_export(const capt_tree* t, capt_grid_info* info, uint8_t* h_cells);

/* Nearest-candidate lists of the clearance (this library's addition; the paper's
 * clearance scans the whole set of the centre's leaf, Lemma 1 case 1).  For every cell
 * of the distance-bound grid (grown by cell / 100) with centre m and half-diagonal rho:
 * the points of the sets of all leaves whose closed cell meets the cell that lie
 * within min(ub, r_max) (1 + 2^-20) + rho of m, each once (in no promised order); ub
 * is the grid's upper bound for the cell.  capt_clearance_fwd with
 * capt_launch_cfg.grid = 1 then answers a centre near the cloud from its cell's list
 * (the FP32 argmin over the list, ties to the lowest point index) instead of the
 * descent and the full set scan: the nearest point that the paper's scan reports is
 * always in the list, and no other list point can beat it, so the distances and
 * indices are the paper's bit for bit (the argument is in dist_grid.cu).  A cell the
 * grid proves farther than r_max from the cloud has an empty list (r_max, -1).  A cell
 * that meets more than 32 leaves or holds more than 1024 such points (a coarse grid)
 * is a fallback cell: its centres take the paper's path.  Device memory: 8 bytes per
 * cell, 4 per entry (each list padded to a multiple of 4), 16 per point.
 * Needs an uploaded tree with r_min = 0, its replicated sets, and capt_build_grid
 * first (a tree without points, or with r_max = 0, gets no lists and no error);
 * capt_build_grid and capt_upload release the lists (they belong to one grid).
 * Do not call it while work on this tree runs on other streams.  Synchronises
 * `stream`.  Errors: CAPT_E_ARG, CAPT_E_STATE, CAPT_E_RANGE (2^32 entries or more: use
 * a coarser grid), CAPT_E_NOMEM, CAPT_E_BOUNDS (the two walks of the builder
 * disagreed), CAPT_E_CUDA. */
int capt_build_near_lists(capt_tree* t, void* stream);

/* De-duplicated ("compact") affordance sets: Alg. 1 copies a point into the set of
 * every leaf cell that affords it, so the sets replicate the cloud many times over
 * (Sec. VII names compressing or de-duplicating them as the way to larger clouds).  The
 * compact form keeps one copy of the cloud, in Z-order (capt_morton_order) and cut into
 * chunks of 32 consecutive points with their FP32 boxes, and gives each leaf the
 * ascending list of the chunks that hold a point of its set; the leaf box stays the
 * box of its set.  The listed chunks hold a superset of the set inside the cloud, so
 * every flag is unchanged (a point found is a cloud point within r; Lemma 1 puts every
 * such point in the set).  The queries use it with the launch configuration's scan
 * mode CAPT_SCAN_COMPACT; the autotuners include it once it exists.
 * Built on the tree's device from its uploaded sets, the Z-order included (stream-ordered
 * on `stream`, the call synchronises it); about 16 bytes per point plus 32 bytes per
 * leaf plus 4 bytes per list entry.  drop_full = 1 then frees the replicated device
 * sets: edge validation and joint-angle configurations switch to the compact scan by
 * themselves, while the plain and chunked scan modes, clearance (which needs the point
 * of every slot) and the work counters return CAPT_E_STATE until capt_upload runs
 * again; the drop is refused while an edge plan of the tree exists.  capt_upload and
 * capt_free release the compact form.  With drop_full, the caller must make sure that
 * no work queued on other streams still uses the tree (the call synchronises `stream`
 * only).
 * Errors: CAPT_E_ARG, CAPT_E_STATE (not uploaded, or the replicated sets already
 *         dropped), CAPT_E_RANGE (more than 1.6M chunks), CAPT_E_NOMEM, CAPT_E_CUDA. */
int capt_compact(capt_tree* t, int drop_full, void* stream);

/* Build the CAPT on the current CUDA device (Alg. 1, Sec. IV-A/B) from points already
 * in device memory.  The tree is the one capt_build makes from the same points and
 * radii, bit for bit (splits, sets in ascending index, boxes, prune decisions), and it
 * comes back already uploaded to the current device: the query calls can use it at
 * once.  Instead of the recursion with a carried set z, each leaf's set is found
 * directly as the points its closed cell affords (the same set, since the FP64
 * distance only grows as a cell shrinks), the medians come from one sorted order per
 * axis partitioned level by level.
 * d_points: device float[n][3] on the current device, read during the call only.
 * stream: the build's kernels and copies run on it; the call returns when they are
 *   done.  Temporary device memory (about 100 bytes per leaf plus twice the affordance
 *   sets) is allocated and freed inside the call.
 * The host form (capt_stats, capt_export, capt_upload to another device) is copied
 * back from the device the first time one of those calls needs it.
 * Errors: CAPT_E_ARG (out == NULL, d_points == NULL with n > 0, n >= 2^30),
 *         CAPT_E_RANGE (radii, or more than 2^32 point blocks in the sets),
 *         CAPT_E_NONFINITE, CAPT_E_NOMEM, CAPT_E_CUDA. */
int capt_build_device(const float* d_points, size_t n, float r_min, float r_max, void* stream, capt_tree** out);

/* A raw cloud (e.g. one depth frame) to an uploaded tree on the current device in one
 * call: sfc_filter_device at r_filter (Alg. 2), the kept points gathered in the filter's
 * output order, then capt_build_device on them (Alg. 1).  The tree is the one capt_build
 * makes from points[kept] on the host.  d_points: device float[n][3]; d_kept: device
 * uint32[n] (caller-owned) receiving the kept indices (the tree's point i is input point
 * d_kept[i]), or NULL when not wanted; *n_kept (host) their count.  Temporary device
 * memory is allocated and freed inside; the call returns when the tree is complete.
 * Errors: those of sfc_filter_device and capt_build_device. */
int capt_build_frame_device(const float* d_points, size_t n, float r_filter, float r_min, float r_max,
                            uint32_t* d_kept, size_t* n_kept, void* stream, capt_tree** out);

/* One flag per sphere (Alg. 3).  d_centers: device float[m][3]; d_radii: device
 * float[m]; d_flags: device uint8[m] receives 1 = collides, 0 = free.  m = 0 is a
 * no-op.  Errors: CAPT_E_ARG, CAPT_E_STATE, CAPT_E_CUDA. */
int capt_query_spheres(const capt_tree* t, const float* d_centers, const float* d_radii, size_t m,
                       uint8_t* d_flags, void* stream);

/* One flag per configuration of S spheres: 1 iff any sphere collides (Sec. IV-D; a
 * configuration stops being checked at its first colliding sphere).
 * d_centers: device float[C][S][3]; d_radii: device float[S] (sphere s of every
 * configuration has radius d_radii[s]); d_flags: device uint8[C].  1 <= S <= 64.
 * Errors: CAPT_E_ARG, CAPT_E_STATE, CAPT_E_CUDA. */
int capt_query_configs(const capt_tree* t, const float* d_centers, const float* d_radii, size_t C, int S,
                       uint8_t* d_flags, void* stream);

/* capt_query_configs from HOST memory: h_centers float[C][S][3], h_radii float[S],
 * flags to h_flags uint8[C]; the call returns when h_flags is complete (it
 * synchronises `stream`).  When h_centers is page-locked (cudaHostAlloc, torch
 * pin_memory) the kernel reads the centres straight from host memory, each once (on
 * Grace systems over NVLink-C2C), with no staging copy; flags are written the same way
 * when h_flags is page-locked.  Pageable centres are copied in 64 Ki-configuration
 * chunks that overlap with the queries of the previous chunk.  The first call
 * allocates small device buffers (chunk buffers for pageable input), kept by the tree.
 * Errors as capt_query_configs, CAPT_E_NOMEM. */
int capt_query_configs_host(capt_tree* t, const float* h_centers, const float* h_radii, size_t C, int S,
                            uint8_t* h_flags, void* stream);

/* Algorithmic work of capt_query_configs, counted sequentially per configuration (for
 * roofline accounting): d_counts (device uint64[8], below) receives += [spheres examined (up to
 * and including each configuration's first hit), spheres within reach of the cloud's
 * bounding box (these descend), spheres passing their leaf's box test (Alg. 3),
 * affordance points scanned by Alg. 3 alone (in stored order, up to and including the
 * first hit), chunk boxes tested, points scanned in the chunks whose box the sphere
 * reaches (up to and including the first hit)].  The query kernels do the work of
 * entries 0-2, 4 and 5; entry 3 is the plain method's scan for comparison.  The two
 * walks must find the same hits: a disagreement latches CAPT_E_BOUNDS in the device
 * status word.  When the tree's configuration launch has grid = 1 (capt_build_grid),
 * the counts follow that path and d_counts holds two more entries: [6] grid lookups
 * (spheres that reach the cloud's box), [7] spheres the grid decides (a certain miss
 * needs nothing more; a certain hit ends its configuration); only the undecided
 * descend.  d_counts: device uint64[8].  The caller zeroes d_counts.  Errors as
 * capt_query_configs. */
int capt_count_config_work(const capt_tree* t, const float* d_centers, const float* d_radii, size_t C, int S,
                           uint64_t* d_counts, void* stream);

/* capt_count_config_work for capt_query_spheres: m spheres with their own radii
 * (d_radii device float[m]), each counted as a configuration of one sphere; the same
 * eight counters (the grid's when the tree's sphere launch has grid = 1). */
int capt_count_sphere_work(const capt_tree* t, const float* d_centers, const float* d_radii, size_t m,
                           uint64_t* d_counts, void* stream);

/* Leaf index i - (N - 1) reached by the descent of Alg. 3 for each centre.
 * d_centers device float[m][3]; d_leaves device uint32[m].  Diagnostics. */
int capt_query_leaves(const capt_tree* t, const float* d_centers, size_t m, uint32_t* d_leaves, void* stream);

/* Read and clear the device status word (synchronises `stream`): CAPT_OK, or the
 * latched CAPT_E_TIMEOUT / CAPT_E_BOUNDS.  Errors: CAPT_E_ARG, CAPT_E_STATE, CAPT_E_CUDA. */
int capt_device_status(const capt_tree* t, void* stream);

/* ---------------------------------------------------------------------------------
 * Launch configuration and autotuning
 * --------------------------------------------------------------------------------- */

enum { CAPT_STAGE_GLOBAL = 0, /* T read through L1/L2 */
       CAPT_STAGE_SMEM = 1    /* the top levels of T copied to shared memory by a bulk
                                 asynchronous (TMA) copy at block start */ };
enum { CAPT_KERNEL_SPHERES = 0, CAPT_KERNEL_CONFIGS = 1, CAPT_KERNEL_EDGES = 2, CAPT_KERNEL_CLEARANCE = 3,
       CAPT_KERNEL_JOINTS = 4, CAPT_N_KERNELS = 5 };

typedef struct capt_launch_cfg {
    int32_t warps_per_block;   /* 1..16 */
    int32_t spheres_per_lane;  /* tile size.  Spheres: 1, 2, 4 or 8 spheres per lane
                                  (32 x that per warp tile).  Configurations: 2, 4, 8
                                  or 16, for 4, 8, 16 or 32 configurations per warp
                                  tile.  Edges and joint-angle configurations: not
                                  used (one configuration per lane). */
    int32_t staging;           /* CAPT_STAGE_* */
    int32_t chunk;             /* edges: configurations per work item (1..1024, rounded
                                  up to a multiple of 32).  Spheres and configurations:
                                  the affordance scan, CAPT_SCAN_* */
    int32_t prefetch;          /* configurations: 0..CAPT_MAX_PREFETCH.  With k > 0 every
                                  lane asks L2 for its centres of the pass (of 128
                                  spheres) k passes ahead of the one it tests
                                  (prefetch.global.L2), so the loads of the root box test
                                  find them there.  Clearance: a trajectory k x (resident
                                  blocks) ahead per block (cp.async.bulk.prefetch).
                                  0 = none.  Other kernels: must be 0. */
    int32_t grid;              /* sphere, configuration, edge and joint-angle queries:
                                  1 = classify each sphere that reaches the cloud's
                                  bounding box by the tree's distance-bound grid
                                  (capt_build_grid) before any descent: a certain miss is
                                  dropped, a certain hit decides its sphere, configuration
                                  or edge at once, only the undecided descend.  Exact (the
                                  flags do not change).  Ignored while the tree has no
                                  grid.  Clearance: 1 = answer the centres near the cloud
                                  from the nearest-candidate lists
                                  (capt_build_near_lists), with the same results; ignored
                                  while the tree has none.  Default 1 for clearance, 0
                                  for the others. */
} capt_launch_cfg;
#define CAPT_MAX_PREFETCH 4

/* Affordance scan of the sphere and configuration kernels (capt_launch_cfg.chunk). */
enum { CAPT_SCAN_SETS = 0,     /* whole sets, as Alg. 3 */
       CAPT_SCAN_CHUNKED = 1,  /* sets by chunks of 32 points, only those whose box the
                                  sphere reaches (pays when a set's consecutive points are
                                  close in space, as after the filter) */
       CAPT_SCAN_COMPACT = 2   /* the compact sets of capt_compact, chunk boxes first */ };

/* Set / get the launch configuration used for `kernel` on this tree.
 * Errors: CAPT_E_ARG (unsupported value). */
int capt_set_launch_cfg(capt_tree* t, int kernel, const capt_launch_cfg* cfg);
int capt_get_launch_cfg(const capt_tree* t, int kernel, capt_launch_cfg* cfg);

/* Time every supported configuration of the configuration-query kernel on these
 * inputs (CUDA events on `stream`), keep the fastest on the tree and return it.
 * d_flags is overwritten.  best_ms may be NULL.  Synchronises `stream`. */
int capt_autotune_configs(capt_tree* t, const float* d_centers, const float* d_radii, size_t C, int S,
                          uint8_t* d_flags, void* stream, capt_launch_cfg* best, float* best_ms);

/* The same for the sphere-query kernel (capt_query_spheres' arguments). */
int capt_autotune_spheres(capt_tree* t, const float* d_centers, const float* d_radii, size_t m, uint8_t* d_flags,
                          void* stream, capt_launch_cfg* best, float* best_ms);

/* ---------------------------------------------------------------------------------
 * Batched edge validation
 * --------------------------------------------------------------------------------- */

#define CAPT_MAX_JOINTS 16
#define CAPT_MAX_SPHERES 64

/* A serial arm made of spheres.  Joint j rotates its frame about local axis axis[j]
 * (0 = x, 1 = y, 2 = z) by q_j, then the frame origin moves by link[j] expressed in
 * the rotated frame.  Sphere s belongs to link sphere_link[s]: its centre is the
 * origin of that link (before the link's translation) plus R * sphere_offset[s], with
 * R the rotation after joint sphere_link[s].  All FP32; sin and cos are the library's
 * own Cody-Waite-reduced Taylor polynomials, so results do not depend on libm. */
typedef struct capt_arm {
    int32_t n_joints;                          /* 1..CAPT_MAX_JOINTS */
    int32_t n_spheres;                         /* 1..CAPT_MAX_SPHERES */
    float base[3];
    int32_t axis[CAPT_MAX_JOINTS];
    float link[CAPT_MAX_JOINTS][3];
    int32_t sphere_link[CAPT_MAX_SPHERES];
    float sphere_offset[CAPT_MAX_SPHERES][3];
    float sphere_radius[CAPT_MAX_SPHERES];
} capt_arm;

enum { CAPT_EDGES_PERSISTENT = 0, /* one persistent launch over (edge, chunk) work items */
       CAPT_EDGES_PER_EDGE = 1    /* one launch per edge (baseline) */ };

/* Validate E straight joint-space edges: edge e holds the n_e configurations
 * q_k = q_a + (k / (n_e - 1)) (q_b - q_a), k = 0..n_e-1 (q_a alone when n_e = 1), and
 * is valid iff none of them collides (Sec. IV-D early termination; an edge stops being
 * checked once one configuration collides).  n_e <= 0 means no configuration: valid.
 * d_qa, d_qb: device float[E][n_joints]; d_nsteps: device int32[E];
 * d_valid: device uint8[E] receives 1 = valid, 0 = collides.
 * Each buffer must hold E entries: the call sees only their base addresses.
 * arm: host pointer, copied.  mode: CAPT_EDGES_*.  CAPT_EDGES_PER_EDGE reads d_nsteps
 * back to the host (it synchronises `stream` once).  Uses scratch owned by the tree, so
 * calls on one tree must not overlap on different streams (an edge plan, which owns
 * its scratch, can run beside them).  In persistent mode the work is counted in items
 * of up to 32..1024 configurations; a batch of more than 2^31 items (2^36 or more
 * configurations) is refused on the device: every edge is reported as not valid (0)
 * and capt_device_status returns CAPT_E_BOUNDS.
 * Errors: CAPT_E_ARG, CAPT_E_STATE, CAPT_E_CUDA, CAPT_E_NOMEM. */
int capt_validate_edges(capt_tree* t, const capt_arm* arm, const float* d_qa, const float* d_qb,
                        const int32_t* d_nsteps, size_t E, uint8_t* d_valid, int mode, void* stream);

/* The same validation as capt_validate_edges in persistent mode, for callers that
 * cannot let the library allocate device memory: a planner in a real-time control loop
 * must not enter the CUDA allocator (cudaMalloc/cudaFree can synchronise the device and
 * take unbounded time), and an application whose device memory belongs to another
 * allocator (a caching allocator or a fixed arena) cannot have raw allocations appear
 * behind its back.  The paper has no counterpart: this is a deployment variant.
 * Instead of a buffer it allocates, the call uses one fixed scratch array inside the
 * library (CAPT_STATIC_MAX_EDGES + 64 words, about 256 KB), which every device that
 * loads the library's device code holds until its context ends.  It calls no allocator.
 *  - E must be <= CAPT_STATIC_MAX_EDGES, else CAPT_E_ARG.
 *  - The first call on a device looks the array's device address up (once per device
 *    and context, with that device current; again after a cudaDeviceReset replaced the
 *    context).  With CUDA's lazy module loading that first call may also load the
 *    library's device code, which is when the array is reserved.  Make that first call
 *    before any stream capture.
 *  - Every call reuses the same array and re-initialises what must start at zero, so
 *    calls whose work overlaps on the GPU (other streams, other host threads) race:
 *    order them on one stream or synchronise between them.
 * Arguments, results and the other errors as capt_validate_edges. */
#define CAPT_STATIC_MAX_EDGES 65536
int capt_validate_edges_static(const capt_tree* t, const capt_arm* arm, const float* d_qa, const float* d_qb,
                               const int32_t* d_nsteps, size_t E, uint8_t* d_valid, void* stream);

/* One flag per configuration given by its joint angles: the arm's kinematics run
 * inside the kernel (the same FP32 chain and sin/cos as the edge validator, one lane
 * per configuration) and each sphere centre is tested as it appears, so the sphere
 * centres never exist in memory.  Flag = 1 iff any sphere collides (Sec. IV-D: a
 * configuration stops being checked at its first colliding sphere); the flags equal
 * those of capt_query_configs on the centres that kinematics gives.
 * d_q: device float[C][arm->n_joints]; d_flags: device uint8[C]; arm: host pointer,
 * copied.  C = 0 is a no-op.  Errors: CAPT_E_ARG, CAPT_E_STATE, CAPT_E_CUDA. */
int capt_query_joint_configs(const capt_tree* t, const capt_arm* arm, const float* d_q, size_t C,
                             uint8_t* d_flags, void* stream);

/* Time every supported launch configuration of capt_query_joint_configs (warps per
 * block x staging) on these inputs, keep the fastest on the tree and return it.
 * d_flags is overwritten; best_ms may be NULL.  Synchronises `stream`. */
int capt_autotune_joint_configs(capt_tree* t, const capt_arm* arm, const float* d_q, size_t C, uint8_t* d_flags,
                                void* stream, capt_launch_cfg* best, float* best_ms);

/* A captured CUDA graph of the persistent edge validator for fixed buffers: one
 * capt_edge_plan_launch replays {work-counter reset, per-edge prefix of work items,
 * persistent kernel} with a single cudaGraphLaunch.  cfg = NULL autotunes the
 * launch configuration (warps per block, spheres per lane, staging, chunk) on the given
 * inputs first, which runs the validator several times on `stream`.  The plan owns
 * its scratch; buffers must outlive it.  Errors as capt_validate_edges. */
typedef struct capt_edge_plan capt_edge_plan;
int capt_edge_plan_create(capt_tree* t, const capt_arm* arm, const float* d_qa, const float* d_qb,
                          const int32_t* d_nsteps, size_t E, uint8_t* d_valid, const capt_launch_cfg* cfg,
                          void* stream, capt_edge_plan** out);
int capt_edge_plan_launch(capt_edge_plan* p, void* stream);
/* The plan's launch configuration and, when it was autotuned, the best time (else 0). */
int capt_edge_plan_info(const capt_edge_plan* p, capt_launch_cfg* cfg, float* tuned_ms);
/* Configurations the plan's last launch evaluated (its warps ran their interpolation,
 * kinematics and sphere tests; an edge stops being evaluated once one collides, so this
 * is at most the sum of n_e), for work accounting.  Synchronous: call it after the
 * launch's stream has finished.  Errors: CAPT_E_ARG, CAPT_E_CUDA. */
int capt_edge_plan_work(const capt_edge_plan* p, uint64_t* configs_evaluated);
void capt_edge_plan_free(capt_edge_plan* p);

/* ---------------------------------------------------------------------------------
 * Differentiable clearance (tree built with r_min = 0)
 * --------------------------------------------------------------------------------- */

/* Forward: for T trajectories x W waypoints x S spheres,
 *   d = min(||c - p*||, r_max) with p* the nearest cloud point: exact whenever the
 *       nearest point is within r_max, because every such point is in the leaf's set
 *       (Lemma 1, case 1); the distance is sqrt of the FP32 squared distance; with
 *       nearest-candidate lists (capt_build_near_lists, grid = 1) the same values come
 *       from the centre's grid cell instead of its leaf set;
 *   cost_t = sum over its W*S spheres of max(0, r_s + margin - d)^2.
 * d_centers device float[T][W][S][3]; d_radii device float[S]; d_cost device
 * float[T]; d_dist device float[T*W*S]; d_argmin device int32[T*W*S] receives the
 * index of p* (lowest index among FP32 ties), or -1 where d = r_max.  1 <= S <= 64,
 * 1 <= W.  The cost sums in a fixed order (bitwise reproducible).
 * Errors: CAPT_E_ARG, CAPT_E_STATE (r_min > 0 or not uploaded), CAPT_E_CUDA. */
int capt_clearance_fwd(const capt_tree* t, const float* d_centers, const float* d_radii, size_t T, int W, int S,
                       float margin, float* d_cost, float* d_dist, int32_t* d_argmin, void* stream);

/* Backward: d_grad_centers[t,w,s,:] = g_t * (-2 h) * (c - p*) / d with
 * h = max(0, r_s + margin - d), when h > 0, d < r_max and d > 0; else 0.
 * d_grad_cost device float[T] (g).  Other arguments as in the forward, whose d_dist and
 * d_argmin it reads.  Errors as capt_clearance_fwd. */
/* Time every supported launch configuration of the clearance forward on these inputs
 * (warps per block, staging, prefetch, and the nearest-candidate lists when the tree
 * has them; CUDA events on `stream`), keep the fastest on the tree and return it.  The
 * outputs are overwritten (every configuration computes the same values).  best_ms may
 * be NULL.  Synchronises `stream`.  Errors as capt_clearance_fwd, and CAPT_E_ARG for
 * T = 0. */
int capt_autotune_clearance(capt_tree* t, const float* d_centers, const float* d_radii, size_t T, int W, int S,
                            float margin, float* d_cost, float* d_dist, int32_t* d_argmin, void* stream,
                            capt_launch_cfg* best, float* best_ms);

int capt_clearance_bwd(const capt_tree* t, const float* d_centers, const float* d_radii, const float* d_dist,
                       const int32_t* d_argmin, const float* d_grad_cost, size_t T, int W, int S, float margin,
                       float* d_grad_centers, void* stream);

/* Algorithmic work of capt_clearance_fwd on m = T x W x S sphere centres (d_centers
 * device float[m][3]), counted sequentially per sphere, for roofline accounting:
 * d_counts device uint64[8] receives += [spheres, spheres within r_max of the cloud's
 * bounding box, spheres whose leaf box is within r_max (Alg. 3's box test at r_max),
 * points of their sets (each scanned in full: the nearest point is wanted, Lemma 1
 * case 1), 4-point blocks of those sets, then three list counts].  When the tree has
 * nearest-candidate lists and its clearance launch has grid = 1 the counts follow that
 * path: the near spheres look up their cell, [5] those answered by a list (an empty one
 * included), [6] list entries scanned (padding included), [7] those of fallback cells,
 * and entries 2-4 count the descents and scans of the fallback spheres only; otherwise
 * [5]-[7] stay 0 and every near sphere descends.  The caller zeroes d_counts.
 * Errors as capt_clearance_fwd. */
int capt_count_clearance_work(const capt_tree* t, const float* d_centers, size_t m, uint64_t* d_counts,
                              void* stream);

#ifdef __cplusplus
}
#endif
#endif /* CAPT_H */
