/*
 * psf.h -- C ABI of the progressive spatio-temporal filtering hot path (B300, sm_103a).
 *
 * One table per render session holds a sparse spatio-directional field: for every
 * basis function (cell) the per-iteration fixed-point accumulators, the cumulative
 * counter c_old and the approximant L~ (Pantaleoni, "Online path sampling control
 * with progressive spatio-temporal filtering", Section "Progressive Spatio-Temporal
 * Filtering").  Each iteration:
 *
 *   psf_insert    scatter path vertices into their cells         (eq. 5-6, Alg. 1)
 *   psf_update    blend each touched cell into its approximant   (eq. 10-11)
 *   psf_query_cv  apply the approximant as a control variate     (Section "Control variates")
 *
 * Conventions shared by every call
 *   - All pointers named d_* are device pointers on the current CUDA device; h_* are
 *     host pointers.  The caller owns every buffer it passes, including the table
 *     memory given to psf_create; the library owns only a small host-side header per
 *     table (and its mapped status word, from a process-wide pool), each batch's
 *     descriptor buffers, and the fixed array of psf_batch_step_noalloc.
 *   - `stream` is a cudaStream_t passed as void* (NULL = the legacy default stream).
 *     Calls enqueue work on it and return without waiting, except psf_export and
 *     psf_get_stats, which synchronise that stream.  psf_create and psf_destroy make no
 *     allocation that synchronizes the device (the first psf_create of a process allocates
 *     a slab of mapped status words).
 *   - Return value: PSF_OK (0) or a negative PSF_ERR_* code for errors detected on the
 *     host (nothing is enqueued then).  Conditions detected on the device set sticky
 *     bits (PSF_STATUS_*) in the table's device status word; psf_update returns them
 *     as last copied back to the host (non-blocking, may lag the device by one call)
 *     and psf_get_stats returns them synchronised.
 *   - Calls on one table must be ordered on one stream (or synchronised by the
 *     caller); tables are independent of each other.
 *
 * Vertex record: 64 bytes = 16 float32, four 16-byte vectors,
 *   v0 = (px, py, pz, w)    position, MIS weight w (eq. 5)
 *   v1 = (nx, ny, nz, tr)   geometric normal, throughput red
 *   v2 = (dx, dy, dz, tg)   incoming ray direction (towards the surface), throughput green
 *   v3 = (Lr, Lg, Lb, tb)   the vertex's value L-bar (eq. 3 / 9), throughput blue
 * The outgoing direction is omega_o = -d (Alg. 1).  t = (tr, tg, tb) is f*cos*w/p to the
 * next vertex of the path.  Vertex arrays must be 16-byte aligned.  For queries the
 * array is depth-major: record j*P + p is vertex j of path p.
 *
 * Cell key (Section "Basis functions and data structures: spatio-directional hashing":
 * a grid over position times a grid over omega_o; the dominant-axis normal bin is an
 * optional extra field).  Packed in 64 bits, bit 63 always 0:
 *   level:2 (61-62, the hierarchy level; see psf_config.levels) | normal bin:3 (58-60) | direction bin:2d (48..) |
 *   x:16 (32-47) | y:16 (16-31) | z:16 (0-15)
 * x = floor(px * 2^q) + 2^15 (likewise y, z); the direction bin is the octahedral map of
 * omega_o on a 2^d x 2^d grid (sgn(0) = +1, lower hemisphere folded outwards, bins
 * clamped to [0, 2^d - 1]), taken in FP32 with correctly rounded operations.
 *
 * Range rule: a vertex is dropped (PSF_STATUS_RANGE, counted in dropped_vertices) if
 * any of p, n, d, L, w is non-finite, d is zero, a cell index leaves [-2^15, 2^15),
 * w < 0, w > 2^15 or |fl32(w * L_c)| > 2^15.  A vertex whose fixed-point weight
 * round(w * 2^F) is 0 carries no weight and is skipped silently (zero_weight_vertices).
 * Sum range: an accepted vertex adds codes of magnitude at most 2^(15+F) (the SH payload's
 * normal moments: below 2^(16+F)), so every sum is exact while fewer than 2^(48-F) vertices
 * (SH payload: 2^(47-F)) are inserted into a table between two updates -- 2^24 at F = 24.
 * The host counts the vertices handed to the inserts (dropped ones included) and sets the
 * sticky PSF_STATUS_SUM_RANGE once an iteration reaches that count; the device adds modulo
 * 2^64 (two's complement), so a sum that does overflow wraps.
 */
#ifndef PSF_H
#define PSF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PSF_OK 0
#define PSF_ERR_INVALID_ARG (-1) /* bad pointer, size, alignment or configuration */
#define PSF_ERR_NO_MEM (-2)      /* table memory or host buffer too small */
#define PSF_ERR_CUDA (-3)        /* a CUDA runtime call failed; see psf_last_cuda_error */
#define PSF_ERR_TOO_MANY (-4)    /* more items than psf_batch_step_noalloc's fixed array holds */

#define PSF_STATUS_TABLE_FULL 1u /* a key found no slot within the probe bound; its vertices were dropped */
#define PSF_STATUS_RANGE 2u      /* at least one vertex failed the range rule */
#define PSF_STATUS_TIMEOUT 4u    /* a bounded device-side wait gave up (batched step) */
#define PSF_STATUS_SUM_RANGE 8u  /* so many vertices were inserted between two updates that a cell's
                                    fixed-point sum may have left the 64-bit range (see the range rule);
                                    sums then wrap modulo 2^64 */

#define PSF_MAX_PROBE 4096u      /* slots a probe visits before declaring the table full */
#define PSF_MAX_BATCH 256u       /* tables per psf_batch_step call */

typedef struct psf_table psf_table;

typedef struct {
    uint32_t log2_capacity; /* slots = 2^log2_capacity, 4..30 */
    uint32_t pos_bits_q;    /* cell size 2^-q in scene units, 0..20 */
    uint32_t dir_bits_d;    /* octahedral direction grid 2^d x 2^d, 0..5 */
    uint32_t use_normal;    /* 1: key includes the dominant-axis normal bin; 0: the paper's 5-d key */
    float alpha_min;        /* 1 / T_max of eq. (11), in [0, 1] */
    float beta;             /* control-variate coefficient (the paper uses [0.5, 1]) */
    uint32_t cv_max_depth;  /* the CV is applied to vertices j < cv_max_depth only */
    uint32_t frac_bits;     /* F: fixed-point fraction bits of the accumulators, 8..32 */
    uint32_t cache_fp16;    /* 1: the update also writes an 8-byte FP16 copy of L~ and queries read it
                               (the blend always keeps the FP32 master, which queries read otherwise) */
    uint32_t blend_mode;    /* 0: eq. (11) square-root blend; 1: constant alpha = alpha_min */
    uint32_t key_layout;    /* where the cell keys live: 1 = a dense 8-byte array, 2 = inside each 64-byte
                               slot record (a probe's key shares the record's 64-byte half with the sums
                               the insert adds to; an FP32 query reads key and approximant from one
                               sector), 0 = 2 for FP32 tables up to 2^22 slots, else 1: the best choice
                               for the probing query (psf_query_cv, psf_step), whose large tables keep
                               more key reads in L2 with the dense array.  With the slot-cache calls
                               (psf_insert_slots + psf_query_cv_slots) 2 was measured faster on every
                               workload.  Results do not depend on it. */
    uint32_t levels;        /* hierarchy levels L, 0..4 (0 and 1: a flat table).  Section "Progressive
                               hierarchical solver": level l has cells 2^l times wider in position
                               (x_l = floor(px * 2^(q-l)) + 2^15, likewise y, z; the same normal and
                               direction bins); every inserted vertex is added to its cell at all L
                               levels, and a vertex at path depth j is read at level min(j, L - 1) by
                               the queries and by psf_insert_progressive (the paper's level choice is a
                               path-footprint heuristic it does not give; the depth stands in for the
                               footprint).  A table holds up to L times the cells of a flat one. */
    uint32_t payload;       /* what a cell holds.  0: RGB (three sums, an RGB approximant).  1: the YCoCg
                               two-band spherical-harmonics payload of Section "Basis functions and data
                               structures: spatio-directional hashing" (last paragraph): luminance in two
                               SH bands over the normal, chroma per cell, so the basis spans normal
                               variation inside a cell.  Per cell and iteration the luminance is fitted by
                               weighted least squares, Y(n) ~ a + g . n (the span of bands 0 and 1),
                               minimising sum w (Y - a - g . n)^2 + sh_ridge * W |g|^2 (W = sum w); chroma
                               (Co, Cg) is the weighted mean; eq. (10)-(11) blend the six coefficients;
                               a query reads the cell's fit at the vertex's own normal, turned back into
                               RGB (R = Y + Co - Cg, G = Y + Cg, B = Y - Co - Cg).  The paper names the
                               representation but not its estimator: the fit is this library's reading,
                               whose band-0 part is eq. (6)'s weighted mean.  Payload 1 needs
                               cache_fp16 = 0, levels <= 1 and key_layout != 2; its cells are 192-byte
                               records plus a dense 8-byte key; it adds |n_k| <= 1 + 2^-10 (unit
                               normals) to the range rule;
                               psf_insert_progressive, psf_export, psf_insert_records,
                               psf_set_approximant and the batched calls reject it
                               (PSF_ERR_INVALID_ARG), psf_export_sh exports it; the slot-cache calls
                               take it (the query then reads the fit at the noted slot). */
    float sh_ridge;         /* payload 1: ridge weight on band 1 relative to the cell's weight, >= 0 and
                               finite (0.01 suggested; 0 allows an unregularised fit, and an iteration
                               whose normal moments leave the system singular then keeps band 1 at 0) */
} psf_config;

/* One exported cell (psf_export), in ascending key order. */
typedef struct {
    uint64_t key;
    int64_t sum[3];       /* this iteration's sum of round(w * L_c * 2^F) (0 after psf_update) */
    int64_t c_new;        /* this iteration's sum of round(w * 2^F) (eq. 5) (0 after psf_update) */
    int64_t c_old;        /* cumulative counter of all blended iterations (eq. 10-11), saturating */
    float L[3];           /* the FP32 approximant */
    uint16_t L_fp16[3];   /* its FP16 copy (IEEE binary16 bits; 0 when cache_fp16 = 0) */
    uint16_t pad;
} psf_cell_record;

/* One exported cell of a table with the SH payload (psf_export_sh), in ascending key order. */
typedef struct {
    uint64_t key;
    int64_t sum[16];  /* this iteration's fixed-point sums (0 after psf_update): Y, Co, Cg, c_new,
                         n_x, n_y, n_z, Y n_x, Y n_y, Y n_z, n_x n_x, n_x n_y, n_x n_z, n_y n_y, n_y n_z,
                         n_z n_z -- each the cell's sum of round(x * 2^F) over its vertices, with x formed
                         in FP32 as w L_c -> YCoCg, w n_k, (w Y) n_k, (w n_j) n_k */
    int64_t c_old;    /* cumulative counter of all blended iterations, saturating */
    float coef[6];    /* a, g_x, g_y, g_z, Co, Cg: luminance a + g . n */
} psf_sh_cell_record;

typedef struct {
    uint64_t capacity;             /* slots */
    uint64_t live_cells;           /* occupied slots */
    uint64_t dropped_vertices;     /* range rule or full table */
    uint64_t zero_weight_vertices; /* skipped: fixed-point weight 0 */
    uint64_t iterations;           /* psf_update calls executed on the device */
    uint32_t status;               /* sticky PSF_STATUS_* bits */
    uint32_t max_probe;            /* longest probe sequence seen by an insert */
    uint64_t table_bytes;          /* psf_table_bytes of the configuration */
    uint64_t touched_cells;        /* cells blended by all psf_update calls so far */
    uint64_t leader_groups;        /* (warp, key) groups that probed and added, all inserts so far
                                      (each issues one bulk reduction of its sums, or four 64-bit
                                      reductions, plus one bitmap reduction); not counted by batched
                                      launches */
} psf_stats;

/* Bytes of device memory a table with this configuration needs (0 if the
 * configuration is invalid).  The caller allocates them (256-byte aligned). */
size_t psf_table_bytes(const psf_config* cfg);

/* Bind a table to caller memory d_mem (>= psf_table_bytes, 256-byte aligned) and
 * enqueue its initialisation (all slots empty, L~ = 0, counters 0) on `stream`.
 * On success *out receives the handle.  d_mem must outlive the table. */
int psf_create(const psf_config* cfg, void* d_mem, size_t bytes, void* stream, psf_table** out);

/* Scatter n vertices (any order) into the table: for each vertex, find or claim its
 * cell and add round(w * L_c * 2^F) to the cell's three sums and round(w * 2^F) to
 * its counter c_new -- eq. (5) and the numerator of eq. (6), in 64-bit fixed point so
 * the result does not depend on the order of the additions.  Several calls may be made
 * per iteration.  n = 0 is a no-op. */
int psf_insert(psf_table* t, const float* d_vertices, uint64_t n, void* stream);

/* Progressive update values (Section "Progressive solver", eq. (9); Alg. 1 and Alg. 2):
 * instead of each vertex's own tail estimate, the value scattered for vertex j comes from
 * the current approximant L~old of the cell of the next vertex of its path (read before
 * this iteration's psf_update).  d_vertices: D*P records, depth-major; v3.xyz is read as
 * the vertex's emitted radiance L_e and t_j as its throughput to vertex j + 1.
 *   field 0 (L~_o, Alg. 1):      value_j = L_e,j + t_j * L~old(x_{j+1})     (last vertex: L_e,j)
 *   field 1 (L~_{o\e}, Alg. 2):  value_j = t_j * (L_e,j+1 + L~old(x_{j+1}))  (last vertex: 0)
 * computed in FP32 from the FP32 approximant (also with cache_fp16), then scattered as
 * psf_insert scatters L = value, except for the range rule: it applies to the vertex's own
 * record (its L_e as the value, and a finite throughput), and the computed value then
 * saturates at |fl32(w * value)| = 2^15 instead of dropping the vertex (a NaN value drops
 * it), so the decision never depends on the precision the value is computed in.  The
 * next-event term that Alg. 2 may add at a vertex is the caller's to add through a plain
 * psf_insert. */
int psf_insert_progressive(psf_table* t, const float* d_vertices, uint32_t P, uint32_t D, uint32_t field,
                           void* stream);

/* End of iteration: every cell with c_new > 0 gets
 *   alpha = max(sqrt(c_new / (c_old + c_new)), alpha_min)        (eq. 11; blend_mode 0)
 *   L~ = (1 - alpha) L~ + alpha * sum / c_new                    (eq. 10)
 *   c_old = c_old + c_new (saturating), sums = c_new = 0,
 * in FP32, plus the FP16 copy when cache_fp16 = 1; untouched cells keep their state.
 * Returns the sticky status bits as last copied back (>= 0, including PSF_STATUS_SUM_RANGE set on the
 * host), or a negative error.  Resets the count of vertices inserted this iteration. */
int psf_update(psf_table* t, void* stream);

/* Control-variate estimate for P paths of depth D (d_vertices: D*P records, depth-major).
 * With C_j the approximant of vertex j's cell (0 when absent; FP16 copy when cache_fp16):
 *   out_j = L_j - beta * t_j * C_{j+1} + beta * C_j   for j < min(D - 1, cv_max_depth)
 *   out_j = L_j                                        otherwise
 * (Section "Control variates", equation CVEstimator: h = t * C_{j+1} is f * L~_i at the
 * next vertex, whose known integral is C_j.)  d_out_rgb receives D*P*3 float32 in the vertex order. */
int psf_query_cv(psf_table* t, const float* d_vertices, uint32_t P, uint32_t D, float* d_out_rgb,
                 void* stream);

/* Biased predictor-corrector estimate (Section "Biased estimation", equation
 * BiasedEstimator: the control variate at beta = 1 with its corrector scaled by gamma):
 *   out_j = gamma * (L_j - t_j * C_{j+1}) + C_j   for j_begin <= j < j_end with j < D - 1
 *   out_j = L_j                                    otherwise
 * gamma = 0 at j_begin = 1, j_end = 2 is the paper's PSTF-B (the approximant replaces the
 * path's estimate at the second vertex); gamma = 1 over all vertices equals psf_query_cv
 * with beta = 1.  Layouts and errors as psf_query_cv; a NaN gamma is PSF_ERR_INVALID_ARG. */
int psf_query_biased(psf_table* t, const float* d_vertices, uint32_t P, uint32_t D, float gamma, uint32_t j_begin,
                     uint32_t j_end, float* d_out_rgb, void* stream);

/* The slot cache (an insert notes where each vertex's query will read):
 * psf_insert_slots is psf_insert of D*P depth-major records (the same table afterwards) that
 * also writes d_slots[i] = the slot of vertex i's cell at the level its query reads (level
 * min(j, levels - 1) at depth j), or PSF_NO_SLOT when the vertex was not added (range rule,
 * zero weight, full table).  psf_query_cv_slots is psf_query_cv over the same records (the
 * same outputs, bit for bit) reading the approximant at d_slots[i] instead of hashing and
 * probing, and probing as usual where d_slots[i] is PSF_NO_SLOT.  The slots stay valid for
 * the table's lifetime (cells never move), so one insert's slots serve the query that
 * follows its update.  d_slots: D*P uint32, caller-owned, 4-byte aligned.  The insert always
 * loads its vertex records directly (vertex_staging bit 0 does not apply). */
#define PSF_NO_SLOT 0xFFFFFFFFu
int psf_insert_slots(psf_table* t, const float* d_vertices, uint32_t P, uint32_t D, uint32_t* d_slots, void* stream);
int psf_query_cv_slots(psf_table* t, const float* d_vertices, const uint32_t* d_slots, uint32_t P, uint32_t D,
                       float* d_out_rgb, void* stream);

/* One whole iteration: psf_insert of the D*P vertices, psf_update, psf_query_cv. */
int psf_step(psf_table* t, const float* d_vertices, uint32_t P, uint32_t D, float* d_out_rgb,
             void* stream);

/* Global counter reset (Section "Temporal averaging", after eq. 11): c_old := 0 in every cell; L~ is kept,
 * so the next update of a cell takes alpha = 1. */
int psf_reset(psf_table* t, void* stream);

/* Copy every occupied cell to h_out in ascending key order.  *n_out receives the number
 * of cells; if it exceeds cap nothing is written and PSF_ERR_NO_MEM is returned.
 * Synchronises `stream`.  Uses a temporary device buffer (stream-ordered allocation). */
int psf_export(psf_table* t, psf_cell_record* h_out, size_t cap, size_t* n_out, void* stream);

/* psf_export for a table with the SH payload (psf_config.payload = 1); other tables return
 * PSF_ERR_INVALID_ARG.  Same conventions as psf_export. */
int psf_export_sh(psf_table* t, psf_sh_cell_record* h_out, size_t cap, size_t* n_out, void* stream);

/* ------------------------------------------------------------------------------------
 * A session sharded across ranks (one GPU each).  Each rank pre-aggregates its share of the
 * vertices in a scratch table and exports the touched cells' fixed-point records; the
 * records travel to the rank that owns their key (owner = (fmix64(key) >> 32) mod ranks);
 * the owner adds them to its table (psf_insert_records; integer sums, so the merged cells
 * are exact under any split of the vertices), blends with psf_update, and the blended cells'
 * approximants travel to the other ranks, which write them into their tables
 * (psf_set_approximant) before answering their own paths' queries.  The arithmetic is that of
 * eq. (5)-(6) and (10)-(11) on one table; only where the additions happen changes.
 * ------------------------------------------------------------------------------------ */

/* One cell's contribution of one iteration: the exported key, sums and c_new of a cell. */
typedef struct {
    uint64_t key;
    int64_t sum[3];
    int64_t c_new;
} psf_record;

/* Add n records (device array, 8-byte aligned, any order; a key may repeat) to the table's
 * current iteration: each key's cell is found or claimed, its sums and c_new are added and
 * it is marked touched, as if the vertices behind the records had been inserted here.  A
 * key with bit 63 set is dropped with PSF_STATUS_RANGE; a full table sets
 * PSF_STATUS_TABLE_FULL.  RGB payload only. */
int psf_insert_records(psf_table* t, const psf_record* d_records, uint64_t n, void* stream);

/* Write the approximant of n cells (d_keys: n uint64, d_L: n*3 float32, device arrays) into
 * the table, finding or claiming each key's cell; counters and sums are left as they are,
 * and the FP16 copy is rewritten when the table keeps one.  Errors as psf_insert_records. */
int psf_set_approximant(psf_table* t, const uint64_t* d_keys, const float* d_L, uint64_t n, void* stream);

/* Synchronised statistics and sticky status.  Synchronises `stream`. */
int psf_get_stats(psf_table* t, psf_stats* out, void* stream);

/* Release the host header (the caller frees d_mem).  All work enqueued on the table must
 * have completed (synchronise its stream first), as for freeing d_mem.  Makes no CUDA call
 * (the table's mapped status word returns to a process-wide pool), so it never waits on the
 * device.  NULL is a no-op. */
int psf_destroy(psf_table* t);

/* Launch knobs of a table's kernels (the autotuner's search space).  Results do not
 * depend on them: the integer sums are order-independent.  psf_create starts from
 * {0, 0, 0, 0, 0, 0, 0} (warp merge, occupancy-limited grids, direct vertex loads, bulk sums,
 * per-path queries);
 * a zero grid cap means the occupancy limit.  A batch (psf_batch_set) copies each table's
 * sum_reduction when its descriptors are set. */
typedef struct {
    uint32_t insert_mode;          /* 0: lanes of a warp holding the same key are merged (runs of
                                      adjacent lanes; any lanes, by match_any, with hierarchy levels)
                                      and one head probes and adds; 1: every vertex adds on its own */
    uint32_t insert_blocks_per_sm; /* cap on resident 256-thread blocks per SM (0 = occupancy limit) */
    uint32_t update_blocks_per_sm;
    uint32_t query_blocks_per_sm;
    uint32_t vertex_staging;       /* bit 0: psf_insert, bit 1: psf_query_cv/_biased stage the vertex
                                      records through shared memory with bulk (TMA) copies, per warp;
                                      a clear bit means direct 16-byte loads */
    uint32_t sum_reduction;        /* how an insert adds a group's three sums and counter to its cell:
                                      0 = one 32-byte bulk reduction from shared memory (TMA),
                                      1 = four 64-bit atomic reductions */
    uint32_t query_layout;         /* how the queries map vertices to threads: 0 = one thread per path,
                                      its vertices walked last to first (also the staged query of
                                      vertex_staging bit 1); 1 = split by depth, one lane per vertex
                                      of a warp tile of 32 / D paths at all D depths, C_{j+1} passed
                                      by a warp shuffle (when D <= 32, else as 0).  Measured on the
                                      B300 (1920x1080, depth 5): 230 vs 255 us -- the per-path walk
                                      keeps a warp's lookups on neighbouring pixels, and the query
                                      is bound by its lookups' DRAM traffic, not by latency */
} psf_launch_config;

/* Set / read the launch knobs of a table (host-side only; affects later calls). */
int psf_set_launch_config(psf_table* t, const psf_launch_config* cfg);
int psf_get_launch_config(const psf_table* t, psf_launch_config* out);

/* ------------------------------------------------------------------------------------
 * Batched iterations: one persistent fused kernel per iteration across many tables.
 *
 * A psf_batch holds device-resident descriptors of up to max_items (table, vertices,
 * output, P, D) items and the words of a grid barrier.  psf_batch_launch runs ONE
 * cooperative kernel (all blocks co-resident) that inserts every item's vertices,
 * waits at a grid barrier, blends every item's touched cells, waits again and answers
 * every item's control-variate query -- the same results, bit for bit, as psf_step on
 * each table alone.  The launch reads only the device descriptors, so it can be
 * captured once in a CUDA graph and replayed while psf_batch_set changes what the
 * descriptors point at (sessions joining and leaving).  Each barrier wait is bounded
 * (barrier_timeout_us); a wait that runs out sets PSF_STATUS_TIMEOUT in the batch and in
 * every item's table, and that iteration's results are undefined.
 * ------------------------------------------------------------------------------------ */

typedef struct {
    psf_table* table;
    const float* d_vertices; /* D*P records, depth-major, 16-byte aligned */
    float* d_out_rgb;        /* D*P*3 float32 */
    uint32_t P;
    uint32_t D;
    uint32_t* d_slots;       /* optional slot cache (D*P uint32, 4-byte aligned): the item's insert
                                notes each vertex's slot there and its query reads it, as
                                psf_insert_slots / psf_query_cv_slots do; NULL = probe */
} psf_batch_item;

typedef struct {
    uint32_t insert_mode;         /* as psf_launch_config.insert_mode */
    uint32_t blocks_per_sm;       /* resident 256-thread blocks per SM (0 = occupancy limit) */
    uint32_t barrier_timeout_us;  /* bound on each grid-barrier wait (0 = 2,000,000) */
    uint32_t test_phantom_blocks; /* testing only: each barrier also waits for this many blocks that
                                     do not exist, so every wait runs out (0 in normal use) */
    uint32_t phase_blocks_per_sm[3]; /* blocks per SM that work in the insert, blend and query phases
                                        (0 = every resident block; the others wait at the next
                                        barrier): fewer warps on a scattered phase contend less for
                                        the same lines.  Results do not depend on them. */
} psf_batch_config;

typedef struct psf_batch psf_batch;

/* Allocate a batch for up to max_items (1..PSF_MAX_BATCH) items: device descriptors and
 * barrier words (cudaMalloc) and a pinned host staging buffer.  cfg may be NULL. */
int psf_batch_create(uint32_t max_items, const psf_batch_config* cfg, psf_batch** out);

/* Enqueue on `stream` the copy of n item descriptors (n <= max_items; n = 0 allowed).
 * Every item's table must have been created on the current device and outlive its use. */
int psf_batch_set(psf_batch* b, const psf_batch_item* items, uint32_t n, void* stream);

/* Enqueue one fused iteration over the items last set (capturable in a CUDA graph). */
int psf_batch_launch(psf_batch* b, void* stream);

/* psf_batch_set followed by psf_batch_launch. */
int psf_batch_step(psf_batch* b, const psf_batch_item* items, uint32_t n, void* stream);

/* Sticky status of the batch (PSF_STATUS_TIMEOUT); synchronises `stream`. */
int psf_batch_status(psf_batch* b, uint32_t* status, void* stream);

/* Release the batch (its work must have completed).  NULL is a no-op. */
int psf_batch_destroy(psf_batch* b);

/* The batched fused iteration without any allocation.  (The paper has no counterpart:
 * this serves callers that cannot allocate device memory on the path that drives the
 * filter -- an application that reserved all device memory in its own pool up front, or
 * a per-frame loop that must not call cudaMalloc/cudaFree because they can synchronize
 * the whole device.)  Same items, results and bounded barrier as psf_batch_step, but the
 * descriptors and barrier words live in a fixed device array inside the library
 * (PSF_NOALLOC_MAX_ITEMS items, about 16 KB), which every GPU that loads the library
 * holds until the process exits; nothing is allocated or freed.  The caller still passes
 * the tables (their memory is the caller's), vertices and outputs.
 *   - n > PSF_NOALLOC_MAX_ITEMS returns PSF_ERR_TOO_MANY (with a message in
 *     psf_last_cuda_error) and enqueues nothing; n = 0 is a no-op.
 *   - The first call on a device resolves the array's device address
 *     (cudaGetSymbolAddress) with that device current.
 *   - Every call on a device shares the one array: the barrier words and the status are
 *     cleared at the start of each call, the descriptors overwritten.  Calls whose work
 *     could overlap on the GPU (different streams without ordering between them) race on
 *     it; order them on one stream or with events.
 *   - A barrier that gives up sets PSF_STATUS_TIMEOUT in every item's table.
 *   - The descriptors are built in a thread-local host buffer and copied from that pageable
 *     memory; to stage such a copy CUDA may wait for earlier work on the stream, so a call
 *     can block the host until that work has finished (psf_batch_set copies from pinned
 *     memory and does not). */
#define PSF_NOALLOC_MAX_ITEMS 64u
int psf_batch_step_noalloc(const psf_batch_item* items, uint32_t n, const psf_batch_config* cfg, void* stream);

/* Text of the last CUDA error seen by this thread's calls (empty if none). */
const char* psf_last_cuda_error(void);

/* ABI version of this header: bump on any incompatible change. */
#define PSF_ABI_VERSION 7
int psf_abi_version(void);

#ifdef __cplusplus
}
#endif

#endif /* PSF_H */
