/*
 * tc.h -- C ABI of libtc.so, a GPU (sm_103a) implementation of the
 * edge-sampled, degree-partitioned triangle counter of Kolountzakis, Miller,
 * Peng and Tsourakakis, "Efficient Triangle Counting in Large Graphs via
 * Degree-based Vertex Partitioning".
 *
 * Problem (Section 1 and Table of symbols): G([n], E) is a simple undirected
 * graph with m edges and t triangles; p is the sparsification parameter.
 * The library
 *   1. keeps every edge independently with probability p (Section 3.1) by a
 *      counter-based hash of the edge and the seed:
 *        keep (u, v), u < v  <=>  (splitmix64(key ^ splitmix64(seed)) >> 11)
 *                                  < floor(p * 2^53),   key = u << 32 | v,
 *      so a given (graph, p, seed) always draws the same sample;
 *   2. splits the vertices of the sampled graph (m_p edges, degrees deg_p)
 *      into heavy (deg_p^2 > m_p) and light (Section 3.2);
 *   3. counts exactly the sampled triangles with at least one light vertex
 *      (t_light) and with three heavy vertices (t_heavy) (Section 3.2);
 *   4. returns estimate = t_light / p^3 + t_heavy / p^3 in float64
 *      (Section 3.1: a triangle survives with probability p^3).
 * With p = 1 the estimate is the exact triangle count.
 *
 * Conventions
 *   - Vertex ids are uint32 in [0, n).  Edge lists are arrays of m uint32
 *     pairs {u0, v0, u1, v1, ...} (row-major m x 2).  Pair order, pair
 *     orientation, repeats and self-loops are all allowed on input; the graph
 *     keeps the canonical simple graph (pairs (min, max), no self-loops, no
 *     repeats), as in Section 4.1.
 *   - Sizes: n < 2^32 - 1 and at most 2^32 - 2 canonical edges.
 *   - Every call returns a tc_status; nothing aborts, traps or prints.  A
 *     failed call leaves its outputs unspecified and the graph usable unless
 *     the status is TC_ECUDA (the CUDA context itself reported an error).
 *   - All device work is stream-ordered on the graph's stream (given at
 *     create; NULL means the legacy default stream).  Calls on one graph must
 *     not overlap; different graphs may be used from different host threads.
 */
#ifndef TC_H
#define TC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    TC_OK = 0,
    TC_EINVAL = 1,   /* bad argument: NULL pointer, p outside (0, 1], endpoint >= n, size limit */
    TC_ENOMEM = 2,   /* device or pinned host allocation failed */
    TC_ECUDA = 3,    /* a CUDA runtime call or kernel launch failed */
    TC_ETIMEOUT = 4, /* a bounded device-side wait gave up (the work was abandoned) */
    TC_EBUSY = 5     /* the object is in use by an unfinished asynchronous call */
} tc_status;

/* Opaque graph: owns the canonical edge list and all scratch on the device. */
typedef struct tc_graph tc_graph;

/* Result of one count.  ms[] holds device times of the phases in
   milliseconds when timing is enabled (tc_graph_set_timing) and the call was
   blocking, else zeros: [0] sample + degrees + partition, [1] orientation +
   CSR build + source buckets, [2] sorted-list intersections, [3] heavy
   block, [4] total.  The work counters give the exact amount of list data
   the intersections read, for bandwidth accounting: every oriented pair
   (a -> b) is resolved by loading the longer of N+(a), N+(b) into an
   on-chip set, a hash set or a bitmap of its rank window (src_elems counts
   those loads), and streaming the shorter one through it (nbr_elems);
   partners counts the pairs. */
typedef struct {
    uint64_t m;         /* canonical edges of the graph */
    uint64_t m_sampled; /* kept edges m_p */
    uint32_t n;         /* vertices */
    uint32_t n_heavy;   /* vertices with deg_p^2 > m_p */
    uint64_t t_light;   /* sampled triangles with >= 1 light vertex */
    uint64_t t_heavy;   /* sampled triangles with 3 heavy vertices */
    double estimate;    /* t_light / p^3 + t_heavy / p^3 */
    uint64_t src_elems; /* list elements loaded into the on-chip sets */
    uint64_t nbr_elems; /* list elements streamed through them */
    uint64_t partners;  /* oriented pairs resolved */
    uint64_t heavy_mma_flops; /* executed tensor-core flops of the dense heavy block and,
                                 when the count uses it, the dense core (0 when neither runs) */
    float ms[8];
} tc_result;

/* Optional device allocator used for every device allocation the library
   makes (for example a framework's caching allocator).  alloc returns NULL
   on failure.  Pass NULLs to restore the default: a stream-ordered memory
   pool of the library's own per device (cudaMallocFromPoolAsync /
   cudaFreeAsync on the graph's stream, or cudaMalloc / cudaFree where no pool
   can be made).  Not thread-safe with concurrent graph creation/destruction. */
typedef void *(*tc_alloc_fn)(uint64_t bytes, void *stream, void *ctx);
typedef void (*tc_free_fn)(void *ptr, void *stream, void *ctx);
void tc_set_allocator(tc_alloc_fn alloc, tc_free_fn free_fn, void *ctx);

/* The default pool keeps the memory of destroyed graphs for the next ones.
   This synchronizes the current device and returns that memory to the
   system.  TC_ECUDA on a CUDA error. */
tc_status tc_release_cached_memory(void);

/* Failure detection of the device-side waits.  Every wait of the tensor-core
   kernels on an mbarrier gives up after a time limit, sets an error bit
   (TC_ETIMEOUT for the count) and lets the kernel release what it holds and
   return, so the context stays usable.  This runs that same wait, for
   limit_us microseconds (1 .. 10^6), on a barrier that nothing arrives at,
   in one small kernel on the current device.  Returns TC_ETIMEOUT when the
   wait gave up (the expected outcome), TC_OK if it completed (a defect),
   TC_EINVAL for a limit out of range, TC_ECUDA on a CUDA error. */
tc_status tc_check_bounded_wait(uint32_t limit_us);

/*
 * Build a graph from m_in uint32 pairs (Section 4.1 canonical simple graph).
 *   edges           m_in pairs; host memory (edges_on_device = 0, any host
 *                   memory, pinned is fastest) or device memory of the
 *                   current device (edges_on_device = 1).  Borrowed: the
 *                   library copies what it needs before returning.
 *   n               number of vertices; every endpoint must be < n.
 *   cuda_stream     cudaStream_t for all work of this graph (NULL = default).
 *   out             receives the graph (NULL on failure).
 * Errors: TC_EINVAL for NULL out, NULL edges with m_in > 0, n == 0, n or m
 * beyond the size limits, an endpoint >= n (nothing stays allocated);
 * TC_ENOMEM; TC_ECUDA.  Blocks until the graph is ready.
 * For graphs of at least 2^25 edges, creation also measures the probe work
 * of a p = 1 count among the top ranks and, where it pays, keeps a dense
 * core of the top 8192 to 65536 ranks (2 K^2 bytes of device memory) whose
 * triangles the tensor cores count; each count decides from its p whether
 * and at what size to use it.  The counts do not depend on that choice.
 */
tc_status tc_graph_create(const uint32_t *edges, uint64_t m_in, uint32_t n, int edges_on_device,
                          void *cuda_stream, tc_graph **out);

/* NULL-safe.  Waits for the graph's pending work, then frees everything. */
void tc_graph_destroy(tc_graph *g);

uint64_t tc_graph_num_edges(const tc_graph *g);    /* canonical m */
uint32_t tc_graph_num_vertices(const tc_graph *g); /* n */
uint64_t tc_graph_device_bytes(const tc_graph *g); /* device memory held */

/* Record per-phase device times (adds CUDA event records to every count).
   Blocking counts report them in tc_result.ms; every count, blocking or
   asynchronous, also leaves them in a ring of TC_TIMING_RING entries that
   tc_graph_timing_drain reads. */
#define TC_TIMING_RING 256
tc_status tc_graph_set_timing(tc_graph *g, int on);

/* The sampled in-degrees of a count are computed only for the vertices whose
   full degree^2 exceeds a lower bound m_lo on the number of kept edges m_p
   (by default p m - (120 p m)^(1/2) - 1, or m at p = 1; a sample below it
   has probability under e^-60).  A sample that still falls below m_lo is
   counted exactly by a fallback that computes every in-degree.  This sets
   m_lo for the graph's later counts (m_lo >= 0), or restores the default
   (m_lo < 0): for diagnostics and tests of both paths (m_lo = 0 makes every
   vertex with an edge a candidate; m_lo > m forces the fallback).  Results
   never depend on it.  TC_EINVAL for a NULL graph. */
tc_status tc_graph_set_sample_floor(tc_graph *g, int64_t m_lo);

/* Which graph the degree partition of Section 3.2 splits, for the graph's
   later counts (and tc_graph_export_sample):
     TC_PARTITION_SAMPLED   (the default) the sampled graph: heavy <=>
                            deg_p^2 > m_p;
     TC_PARTITION_ORIGINAL  the whole graph before sparsification: heavy <=>
                            deg^2 > m, and the sampled triangles are split
                            into t_light / t_heavy by those flags.
   The paper states the partition for "the graph" and runs it on the
   sparsified graph in its hybrid; the second reading is offered as an
   option.  t_light + t_heavy and the estimate are the same under both.
   Batched and served counts always use the sampled graph.  TC_EINVAL for a
   NULL graph or an unknown mode. */
#define TC_PARTITION_SAMPLED 0
#define TC_PARTITION_ORIGINAL 1
tc_status tc_graph_set_partition(tc_graph *g, int mode);

/* The dense core of the top ranks (see tc_graph_create) for the graph's later
   counts: ranks < 0 restores the default (each count chooses from its p),
   0 turns it off, and 8192, 16384, 32768 or 65536 makes every count use a
   core of that many ranks, allocating 2 ranks^2 bytes of device memory if
   creation kept a smaller one (after waiting for the graph's pending work).
   For diagnostics and tests; results never depend on it.  TC_EINVAL for a
   NULL graph, another size, a size above n / 2, or a graph without the dense
   path (fewer than 2^25 edges); TC_ENOMEM if the larger core cannot be
   allocated (the smaller one is already released: later counts run without
   a core until a size that fits is set); TC_ECUDA. */
tc_status tc_graph_set_core_ranks(tc_graph *g, int64_t ranks);

/* Schedule of the intersection kernels of the light class (Section 3.2's
   wedge closures).  Every oriented pair is resolved by its owner, the
   endpoint with the longer out-list (see tc_result); owners are bucketed by
   out-degree d+ into one warp per owner (d+ <= warp_max), a 128-thread block
   per owner (warp_max < d+ <= 1024) and a 1024-thread block per owner
   (d+ > 1024), and an owner's partners are cut into work items.
     warp_max            32 .. 256
     seg_w, seg_b, seg_l most partners per item of the three kernels: powers
                         of two in [64, 1024], [256, 512], [256, 4096]
     work_w, work_b, work_l  an item of an owner with out-degree d holds the
                         largest power of two <= seg partners whose product
                         with d stays <= work (at least 64 or 256 partners);
                         each >= 4096
     run_b               items a mid-owner block takes per grab, 1 .. 8
                         (consecutive items of one owner share its hash set)
     mid_max             owners with warp_max < d+ <= mid_max go to the
                         128-thread blocks, larger ones to the 1024-thread
                         blocks (512 .. 1024)
     lookup              membership test of the block kernels (0 .. 15): bits
                         0 and 2 for the 128-thread blocks, bits 1 and 3 for
                         the 1024-thread blocks.  Bit 0 / 1: a binary search
                         of the owner's sorted row.  Else bit 2 / 3: a bitmap
                         in shared memory of the owner's rank window (from
                         the owner to its largest out-neighbour).  Else a
                         hash set of the owner's list in shared memory.
                         Where the bitmap does not fit the table's memory,
                         the hash set (128-thread blocks) or the binary
                         search (1024-thread blocks); where the set does
                         not fit, the binary search.  The default
                         is 8 (bitmaps for the 1024-thread blocks) on
                         graphs where no window of those owners can exceed
                         their table, else 0.
   Results never depend on the schedule; only the time does.
   tc_graph_set_schedule(g, NULL) restores the default.  TC_EINVAL for a
   NULL graph or a value out of range. */
typedef struct {
    uint32_t warp_max;
    uint32_t seg_w, seg_b, seg_l;
    uint32_t work_w, work_b, work_l;
    uint32_t run_b;
    uint32_t mid_max;
    uint32_t lookup;
} tc_schedule;
tc_status tc_graph_set_schedule(tc_graph *g, const tc_schedule *s);
tc_status tc_graph_get_schedule(const tc_graph *g, tc_schedule *out);
/* Choose the graph's schedule by timing counts at (p, seed): a coordinate
   search over warp_max (64 / 128 / 256), mid_max (512 / 1024), seg_w,
   seg_b (256 / 512), seg_l (1024 / 2048 / 4096) and the membership test
   of each block kernel (hash set, bitmap, binary search), from the current
   schedule, keeping each improvement.  The choice stays with the
   graph; desc (may be NULL) receives it with the strategy of each owner
   bucket.  Runs about 18 x 3 counts; results never depend on it.  On a
   graph with a dense core (tc_graph_create) it then measures the core's
   cost model under the chosen schedule, with two counts each without the
   core and with the allocated one: the probe kernels' rate in streamed list
   entries per second, and the contraction's in flops per second (from the
   time the core adds to the CSR and heavy phases).  Later counts choose
   their core size from these rates instead of the built-in GB300 figures
   (5e11 entries/s, 3.5e15 flop/s).  TC_EINVAL for a NULL graph or p outside
   (0, 1]; TC_ECUDA, TC_ETIMEOUT. */
tc_status tc_graph_autotune(tc_graph *g, double p, uint64_t seed, char *desc, uint32_t desc_len);

/* The dense-core cost model of g: the rates it uses (any pointer may be
   NULL) and the core size in ranks that a count at p chooses by default
   (0: none; tc_graph_set_core_ranks overrides it).  TC_EINVAL for a NULL
   graph or p outside (0, 1]. */
tc_status tc_graph_get_core_model(const tc_graph *g, double p, double *probe_entries_per_s,
                                  double *contraction_flops_per_s, uint32_t *core_ranks);

/* After tc_graph_sync: copy the phase times (8 floats per count, layout of
   tc_result.ms) of the counts completed since the last drain, oldest first,
   at most max_counts of them (older ones beyond the ring are lost).  Returns
   the number of counts written, or -1 on bad arguments / CUDA error. */
int tc_graph_timing_drain(tc_graph *g, float *ms_out, uint32_t max_counts);

/*
 * The hot path: sample with (p, seed), partition, count both classes,
 * rescale (Sections 3.1-3.2).  Blocking: returns when *out is filled.
 * Errors: TC_EINVAL (NULL, p not in (0, 1] or NaN), TC_ECUDA, TC_ETIMEOUT.
 */
tc_status tc_count(tc_graph *g, double p, uint64_t seed, tc_result *out);

/*
 * Same computation, enqueued without waiting.  The result (including the
 * float64 estimate, computed on the device) is written to *out when the
 * stream reaches that point; *out should be pinned host memory
 * (cudaMallocHost) for the copy to be asynchronous.  ms[] is not filled.
 *   cuda_stream  NULL (or the graph's own stream): the count is enqueued on
 *                the graph's stream.  Another cudaStream_t: the count runs
 *                there, after the work already enqueued for the graph, and
 *                the graph's stream waits for it, so tc_graph_sync (or a
 *                synchronisation of cuda_stream) makes *out valid.  The
 *                stream must belong to the graph's device.
 * Counts of one graph share its scratch: they are ordered, never
 * concurrent, whichever streams they are given.
 * Errors: TC_EINVAL (NULL graph or out, p not in (0, 1] or NaN), TC_ECUDA.
 */
tc_status tc_count_async(tc_graph *g, double p, uint64_t seed, tc_result *out, void *cuda_stream);

/*
 * Batched count over graphs already resident (Sections 3.1-3.2 for each
 * graph with its own p[i] and seed[i]).  Graphs with a dense heavy block of
 * their own (2^20 edges or more, see tc_graph_create) are counted on their
 * own path, on their stream after its pending work, so that their heavy
 * class runs on the tensor cores; the other graphs are gathered into one
 * disjoint union on the device (their stored keys, no input is read again)
 * and counted by one launch sequence, their heavy class by the intersection
 * kernels.  out[i] (host memory) receives exactly what tc_count(graphs[i],
 * p[i], seed[i]) returns, except that ms[] is zero, and so are the work
 * counters (src_elems, nbr_elems, partners, heavy_mma_flops) of the graphs
 * counted in the union.
 *   graphs   k graph handles of the current device (a graph may appear more
 *            than once, e.g. with several p); k in 1 .. 65535, at most
 *            2^32 - 2 edges and fewer than 2^32 - 1 vertices in total in
 *            the union.
 * The union's scratch (about 40 bytes per edge) is allocated on a stream of
 * its own and freed before the call returns; it blocks until the results
 * are in out.  The union does not touch the graphs' scratch.
 * Errors: TC_EINVAL (NULL pointers, a NULL graph, p[i] outside (0, 1], size
 * limits), TC_ENOMEM, TC_ECUDA, TC_ETIMEOUT.
 */
tc_status tc_count_batch(tc_graph *const *graphs, const double *p, const uint64_t *seed, uint32_t k,
                         tc_result *out);

/* Wait for all enqueued work of the graph; reports a device-side error or
   timeout raised by that work. */
tc_status tc_graph_sync(tc_graph *g);

/*
 * Choosing p (Section 3.3).  The hybrid's running time is a pass over the
 * m p kept edges plus the triple samples, O((m p)^(3/2) log n / (eps^2 t
 * p^3)); balancing the two gives
 *     p = (m^(1/2) ln n / (t eps^2))^(2/5),
 * clamped to at most 1.  t is a pilot estimate of the triangle count.
 * Returns 1 when t <= 0 (no triangle seen: do not sparsify), -1 for
 * eps <= 0 (or NaN), m == 0 or n < 2.  Host arithmetic only.
 */
double tc_suggest_p(uint64_t m, uint32_t n, double t, double eps);

/*
 * Several counts of one graph in one call (the p-sweep of the paper's
 * remarks in Section 4): count i uses (p[i], seed[i]); they are enqueued
 * back to back on the graph's stream and the call blocks once, at the end.
 * out[i] (host memory) is exactly what tc_count(g, p[i], seed[i]) returns,
 * except ms[].  Errors: TC_EINVAL (NULL pointers, k == 0, a p[i] outside
 * (0, 1]), TC_ENOMEM (pinned staging), TC_ECUDA, TC_ETIMEOUT.
 */
tc_status tc_count_sweep(tc_graph *g, const double *p, const uint64_t *seed, uint32_t k, tc_result *out);

/*
 * Vary p until the estimate stabilises (Section 4, remarks): counts at
 * p_i = min(1, p0 growth^i), i = 0, 1, ... up to p = 1 or max_counts of them
 * (one tc_count_sweep, all with the same seed); the result is the first
 * count i >= 1 whose estimate differs from count i - 1 by at most
 * tol |estimate_i|, else the last one.  *p_used and *counts_used (may be
 * NULL) receive its p and the number of counts run.  Errors: TC_EINVAL
 * (p0 outside (0, 1], growth <= 1, tol < 0 or NaN, max_counts 0 or > 64),
 * and those of tc_count_sweep.
 */
tc_status tc_count_adaptive(tc_graph *g, double p0, double growth, double tol, uint64_t seed, uint32_t max_counts,
                            tc_result *out, double *p_used, uint32_t *counts_used);

/*
 * A pilot count at pilot_p, then the count at tc_suggest_p(m, n,
 * pilot estimate, eps) (Section 3.3), both with seed.  *out is the second
 * count's result (the pilot's when m == 0 or n < 2), *p_used (may be NULL)
 * its p.  Errors: TC_EINVAL (NULL, pilot_p outside (0, 1], eps <= 0), and
 * those of tc_count.
 */
tc_status tc_count_auto(tc_graph *g, double eps, double pilot_p, uint64_t seed, tc_result *out, double *p_used);

/*
 * Test and inspection entry points (not on the hot path).  They run the
 * sampling and partition of tc_count for (p, seed) and copy intermediate
 * results to host memory:
 *   kept_pairs_host  2 * m_sampled uint32: kept canonical edges in
 *                    canonical (sorted) order; may be NULL.  Must hold
 *                    2 * tc_graph_num_edges(g) uint32.
 *   heavy_host       n bytes, 1 for heavy vertices; may be NULL.
 *   deg_host         n uint32 sampled degrees; may be NULL.
 *   m_sampled        receives m_p; may be NULL.
 */
tc_status tc_graph_export_sample(tc_graph *g, double p, uint64_t seed, uint32_t *kept_pairs_host,
                                 uint8_t *heavy_host, uint32_t *deg_host, uint64_t *m_sampled);

/*
 * The degree-oriented CSR of the sampled graph that the counting kernels
 * use, in the original vertex ids: every kept edge once, directed from the
 * endpoint of lower rank to the higher one, where rank = (degree in the
 * whole graph, id) is fixed when the graph is created; each row lists its
 * out-neighbours in increasing rank.
 *   rowptr_host  n + 1 uint32;  col_host  m_sampled uint32 (capacity m).
 */
tc_status tc_graph_export_csr(tc_graph *g, double p, uint64_t seed, uint32_t *rowptr_host,
                              uint32_t *col_host, uint64_t *m_sampled);

/* The canonical edge list held by the graph (2 * m uint32, sorted). */
tc_status tc_graph_export_edges(tc_graph *g, uint32_t *pairs_host);

/*
 * Batched counting: k independent graphs resident together and counted by
 * one launch (a CUDA graph captured on the first tc_batch_count and replayed
 * afterwards).  Every graph gets exactly the result that
 * tc_graph_create + tc_count would give it (same sample, partition,
 * classes and estimate); the batch only changes how the work is launched.
 * The dense tensor-core path of the heavy class is not used in batches (the
 * intersection kernels count that class).
 *
 * tc_batch_create
 *   edges         the graphs' pair lists concatenated (graph 0 first), each
 *                 in its own local ids [0, n_g); host or device memory
 *                 (edges_on_device); same input rules as tc_graph_create.
 *   m_per_graph   k pair counts; n_per_graph  k vertex counts (each >= 1).
 *   k             1 .. 65535 graphs; sum of n_g below 2^32 - 1 and at most
 *                 2^32 - 2 canonical edges in total.
 *   cuda_stream   stream for all work (NULL: the batch creates its own).
 * Errors: TC_EINVAL (bad sizes, an endpoint >= its n_g), TC_ENOMEM, TC_ECUDA.
 *
 * tc_batch_count  p[k], seed[k] per graph; out[k] results (host memory).
 * Blocking.  TC_EINVAL if any p is outside (0, 1].
 */
typedef struct tc_batch tc_batch;
tc_status tc_batch_create(const uint32_t *edges, const uint64_t *m_per_graph, const uint32_t *n_per_graph, uint32_t k,
                          int edges_on_device, void *cuda_stream, tc_batch **out);
tc_status tc_batch_count(tc_batch *b, const double *p, const uint64_t *seed, tc_result *out);

/*
 * Autotune the batch's intersection schedule (see tc_schedule): a coordinate
 * search, one axis at a time, timing each candidate on this batch with these
 * (p, seed): the owners' split between one warp and one block (warp_max 64 /
 * 128 / 256), between the 128- and 1024-thread blocks (mid_max 512 / 1024),
 * the work-item sizes of the warp and mid-owner kernels, and the membership
 * test of each block kernel (a shared-memory hash set, a shared-memory bitmap
 * of the owner's rank window, or a binary search of the owner's sorted row).  The fastest is kept for the batch's later counts
 * and remembered for batches of the same shape (log2 of edges, vertices,
 * graphs and average degree) created later in this process.  Counts are
 * identical under every schedule.  desc (may be NULL) receives the choice,
 * with the strategy of each owner bucket.
 */
tc_status tc_batch_autotune(tc_batch *b, const double *p, const uint64_t *seed, char *desc, uint32_t desc_len);
void tc_batch_destroy(tc_batch *b); /* NULL-safe */
uint32_t tc_batch_size(const tc_batch *b);
uint64_t tc_batch_num_edges(const tc_batch *b);    /* canonical edges of all graphs */
uint64_t tc_batch_device_bytes(const tc_batch *b);

/*
 * Serving: count requests (graph, p, seed) as they arrive, with continuous
 * batching.  The paper states the problem for one graph and one (p, seed)
 * at a time (Sections 1 and 3.1); the server only changes how many such
 * problems share a launch, never a result: every request gets exactly what
 * tc_graph_create + tc_count on its graph would return.
 *
 * Graphs are registered once (tc_server_add_graph) and kept resident in
 * device memory as canonical edge lists, with a pinned host copy.  A
 * worker thread owns `slots` count slots, each with its own stream and
 * scratch for a union of up to slot_edges edges, slot_vertices vertices and
 * slot_requests requests.  Whenever a slot is free and requests are queued,
 * the worker admits the longest prefix of the queue (first come, first
 * served) that fits the slot and whose graphs are (or can be made)
 * resident, gathers their edge lists into the slot's union and runs the
 * batched count there; requests that arrive meanwhile wait for the next
 * free slot, and the slots' counts overlap on the device.
 *
 * HBM budget: slot scratch plus resident graphs (16 bytes per canonical
 * edge) never exceed budget_bytes.
 * A graph that is not resident when a request needs it is uploaded again
 * from its host copy, first evicting the least recently used graphs that no
 * slot is using; if that still leaves no room, the request waits in the
 * queue until running counts release their graphs.
 *
 * tc_server_create
 *   budget_bytes   device bytes the server may hold (slots + graphs)
 *   slots          1 .. 8
 *   slot_edges     canonical edges of one slot's union (>= 1)
 *   slot_vertices  vertices of one slot's union (1 .. 2^32 - 2)
 *   slot_requests  requests of one slot's union (1 .. 65535)
 * Errors: TC_EINVAL (bad sizes), TC_ENOMEM (the slots alone exceed the
 * budget, or an allocation failed), TC_ECUDA.
 *
 * tc_server_add_graph  edges as for tc_graph_create (host or device
 *   memory, local ids [0, n), repeats and self-loops allowed); blocks until
 *   the graph is canonical and stored; *gid receives its id.  TC_EINVAL
 *   also when the graph alone exceeds a slot's edge or vertex capacity,
 *   TC_ENOMEM when it exceeds the budget left after the slots.
 *
 * tc_server_submit  queue one request; returns at once with *ticket.
 *   TC_EINVAL for an unknown gid or p outside (0, 1].
 *
 * tc_server_poll  TC_OK: the request is done and *info holds its result
 *   (info->status is its own status; the ticket is then released);
 *   TC_EBUSY: still queued or running; TC_EINVAL: unknown ticket.
 * tc_server_wait  as poll, blocking up to timeout_ms (TC_EBUSY after it).
 *
 * Times in tc_request_info are microseconds since tc_server_create on the
 * host's steady clock: t_submit when submit was called, t_admit when its
 * slot launch was enqueued, t_done when the worker saw that launch finish.
 */
typedef struct tc_server tc_server;
typedef struct {
    tc_result res;       /* ms[] is zero */
    int32_t status;      /* tc_status of this request */
    uint32_t wave_size;  /* requests counted in the same slot launch */
    double t_submit_us, t_admit_us, t_done_us;
} tc_request_info;
typedef struct {
    uint64_t submitted, completed, queued;  /* queued: submitted, not yet admitted */
    uint64_t waves, max_wave;               /* slot launches; most requests in one */
    uint64_t resident_graphs, resident_bytes, graphs;
    uint64_t slot_bytes, budget_bytes;
    uint64_t uploads, evictions;            /* re-uploads after eviction; evictions */
} tc_server_stats;
tc_status tc_server_create(uint64_t budget_bytes, uint32_t slots, uint64_t slot_edges, uint32_t slot_vertices,
                           uint32_t slot_requests, tc_server **out);
tc_status tc_server_add_graph(tc_server *srv, const uint32_t *edges, uint64_t m_in, uint32_t n, int edges_on_device,
                              uint32_t *gid);
tc_status tc_server_submit(tc_server *srv, uint32_t gid, double p, uint64_t seed, uint64_t *ticket);
tc_status tc_server_poll(tc_server *srv, uint64_t ticket, tc_request_info *info);
tc_status tc_server_wait(tc_server *srv, uint64_t ticket, uint32_t timeout_ms, tc_request_info *info);
tc_status tc_server_get_stats(tc_server *srv, tc_server_stats *out);
/* Stops the worker after the requests already admitted finish; queued ones
   are dropped.  NULL-safe. */
void tc_server_destroy(tc_server *srv);

/*
 * Count without allocating (the paper has no counterpart: this exists for
 * callers that cannot allocate device memory, such as a host framework
 * whose memory pool already owns the GPU, or code where a device allocation
 * would synchronise the device or is not permitted).  Same computation and
 * result as tc_graph_create + tc_count + tc_graph_destroy, for graphs of at
 * most TC_NOALLOC_MAX_EDGES input pairs and TC_NOALLOC_MAX_VERTICES
 * vertices; larger inputs return TC_EINVAL.
 *   edges_dev    m_in uint32 pairs in device memory of the current device
 *                (any order, repeats and self-loops allowed, as in create).
 *   out_host     receives the result (host memory); ms[] is zero.
 *   cuda_stream  stream for the work (NULL = default); the call blocks
 *                until the result is in *out_host.
 * All scratch lives in one fixed __device__ array inside the library
 * (about 24 MiB), held by every GPU that loads it until the process exits.
 * The first call on a device looks up that array's device address (kept for
 * the process; a device reset between calls is not supported).  Calls
 * share the array (each
 * clears what must start at zero), so calls that overlap on the GPU race:
 * serialise them.  Nothing is allocated: no cudaMalloc, no cudaFree, no
 * allocator callback.
 */
#define TC_NOALLOC_MAX_EDGES (1ull << 18)
#define TC_NOALLOC_MAX_VERTICES (1u << 18)
tc_status tc_count_noalloc(const uint32_t *edges_dev, uint64_t m_in, uint32_t n, double p, uint64_t seed,
                           tc_result *out_host, void *cuda_stream);

/*
 * Triple sampling (Section 3.2), on the sample of Section 3.1 (the hybrid
 * algorithm of Section 3.3 when p < 1): the "Simple" and "Hybrid" columns
 * of the paper's experiments.  The edge sample is the one tc_count draws
 * for (p, seed).  On the sampled graph, U is a set of vertex triples that
 * holds every triangle, taken vertex by vertex in id order with neighbour
 * lists sorted by id:
 *   TC_TRIPLES_SIMPLE  every vertex contributes its wedges: the C(d, 2)
 *                      pairs {N(u)[a], N(u)[b]}, a < b, numbered
 *                      b (b - 1) / 2 + a;
 *   TC_TRIPLES_HYBRID  light vertices (deg_p^2 <= m_p) contribute their
 *                      wedges, heavy ones their 2-paths u - v - w (v in
 *                      N(u), w in N(v), numbered by v's position, then w's):
 *                      sum over v in N(u) of deg_p(v) of them.
 * A wedge v-u-w is a triangle iff vw is an edge; a 2-path iff w != u and uw
 * is an edge.  Every triangle is in U once per light corner and twice per
 * heavy corner.  Sample i (0 <= i < s) is the triple of index
 * floor(h_i |U| / 2^64), h_i = splitmix64(i ^ splitmix64(~seed)): s
 * independent uniform draws.  estimate = |U| (2 closed_wedge +
 * closed_path) / (6 s) / p^3 in float64, an unbiased estimate of t.
 *   samples   s; 0 draws m_p samples (as many queries as kept edges).
 *   out       host memory; ms is the device time of the call.
 * The first call on a graph builds and keeps the symmetric adjacency of the
 * whole graph in original ids (8 m + 4 n bytes); every call uses 12 m +
 * 12 n bytes more of scratch, also kept for later calls (released by
 * tc_graph_destroy).  Blocks until *out is filled.
 * Errors: TC_EINVAL (NULL graph or out, p outside (0, 1], an unknown mode,
 * graphs of 2^31 edges or more), TC_ENOMEM, TC_ECUDA.
 */
#define TC_TRIPLES_SIMPLE 0
#define TC_TRIPLES_HYBRID 1
typedef struct {
    uint64_t m, m_sampled;
    uint32_t n, n_heavy;   /* n_heavy: vertices whose triples are 2-paths (0 in the simple mode) */
    uint64_t universe;     /* |U| */
    uint64_t samples;      /* s */
    uint64_t closed_wedge; /* sampled wedges that are triangles */
    uint64_t closed_path;  /* sampled 2-paths that are triangles */
    double estimate;
    uint32_t mode;         /* TC_TRIPLES_SIMPLE or TC_TRIPLES_HYBRID */
    float ms;
} tc_triple_result;
tc_status tc_count_triples(tc_graph *g, double p, uint64_t seed, uint64_t samples, int mode, tc_triple_result *out);

/*
 * Semi-streaming count (Section 5.2) for graphs whose edges stay in host
 * memory: three passes over an adjacency-list stream, with only vertex
 * arrays, the samples and a query table on the device.
 *   offsets, adj  host memory: the symmetric adjacency of a simple graph,
 *                 offsets[n + 1] (offsets[0] = 0) and adj[offsets[n]]; the
 *                 neighbours of u are adj[offsets[u] .. offsets[u + 1]),
 *                 sorted by id, and every edge appears in both endpoints'
 *                 lists (m = offsets[n] / 2).  Pinned memory that is mapped
 *                 into the device is read in place; other host memory is
 *                 copied through the device in chunks of chunk_entries
 *                 (0: 2^26) entries, three times.
 *   Pass 1 finds the heavy vertices as the paper does: stream entry j is
 *   sampled iff (splitmix64(j ^ splitmix64(seed + 1)) >> 11) <
 *   floor(q 2^53), q = min(1, heavy_factor m^(1/2) ln n / (2 m)), both ends
 *   of a sampled entry are candidates, and H = the candidates with
 *   deg^2 > m (a vertex of degree above m^(1/2) is missed with probability
 *   about n^-heavy_factor; one that is missed is simply treated as light).
 *   U holds the wedges of the vertices outside H (C(d, 2) each, in vertex
 *   order, wedge b (b - 1) / 2 + a of the sorted list) and then the pairs
 *   (edge e, H[i]) of every edge (the entries u < v in stream order) with
 *   every vertex of H, index |U_L| + e |H| + i; every triangle is in U three
 *   times.  Sample i is U's triple floor(h_i |U| / 2^64), h_i =
 *   splitmix64(i ^ splitmix64(~seed)); pass 2 reads the samples' list
 *   entries and puts their third edges in a device hash table, pass 3 marks
 *   the queries that are edges of the stream.
 *   estimate = |U| (closed_wedge + closed_pair) / (3 s), an unbiased
 *   estimate of t (given H).
 *   samples       s (0: m), at most 2^30.
 * Blocks; device memory is allocated and freed by the call (about 40 n +
 * 70 s bytes, plus two chunk buffers when the stream is copied).
 * Errors: TC_EINVAL (NULL pointers with data, offsets not starting at 0 or
 * decreasing, an odd or too large offsets[n] (2^33 or more entries), a list
 * that is not sorted, has a self-loop or an id >= n, a stream that is not
 * symmetric, s > 2^30, heavy_factor <= 0), TC_ENOMEM, TC_ECUDA.
 */
typedef struct {
    uint64_t m;
    uint32_t n, n_heavy;      /* n_heavy: |H| */
    uint64_t candidates;      /* distinct ends of the sampled entries */
    uint64_t sampled_entries; /* stream entries sampled in pass 1 */
    uint64_t universe;        /* |U| */
    uint64_t samples;         /* s */
    uint64_t closed_wedge, closed_pair;
    double estimate;
    uint64_t bytes_streamed;  /* adjacency bytes read over the three passes */
    uint32_t passes;
    float ms;
} tc_stream_result;
tc_status tc_stream_count(const uint64_t *offsets, const uint32_t *adj, uint32_t n, uint64_t seed, uint64_t samples,
                          double heavy_factor, uint64_t chunk_entries, void *cuda_stream, tc_stream_result *out);

/* Static description of a status code. */
const char *tc_status_str(tc_status s);

/* Library version, major * 10000 + minor * 100 + patch. */
int tc_version(void);

/* Number of CUDA kernels this library has launched in this process (all
   graphs, all threads); for launch accounting in benchmarks. */
uint64_t tc_launch_count(void);

#ifdef __cplusplus
}
#endif

#endif /* TC_H */
