/*
 * sg2v.h -- C ABI of the B300 colour-coding tree-counting library.
 *
 * Method: SubGraph2Vec (Chen et al., arXiv 2009.11665).  A tree template T
 * with k vertices is counted in a graph G by colouring G's vertices with kc
 * colours and counting *colourful* embeddings (all template vertices get
 * distinct colours, Sec. 2.2.2).  The count comes from a dynamic program over
 * a recursive split of T into an active and a passive child (Sec. 2.3.2,
 * Alg. 2), computed in the decoupled form of Alg. 3 / Eq. 1: per split, a
 * sparse-times-dense product  Y = A * M_passive  (Alg. 4, Alg. 6) and an
 * element-wise multiply-add over colour-set splits
 *   M(v, S) = sum over S_a subset of S, |S_a| = |T_a| of
 *             M_active(v, S_a) * Y(v, S minus S_a)            (Alg. 5 eMA).
 * The root table summed over vertices, divided by alpha (automorphisms of T)
 * and by P (probability that k vertices are colourful) is the estimate of
 * emb(T, G) for one colouring (Alg. 1, finalCount).
 *
 * Conventions shared by every entry point
 *  - Every function returns an sg2v_status; nothing aborts, throws or exits.
 *    sg2v_last_error() gives a human-readable detail of the last failure on
 *    the calling thread.
 *  - Graph and plan handles are opaque and owned by the library; free them
 *    with the matching *_destroy.  The caller owns every array it passes.
 *  - "host or device" arrays may live in host memory (pageable or pinned) or
 *    in device memory of the current device; the library inspects the pointer
 *    and copies as needed (host inputs and outputs make the call include the
 *    host<->device copies).
 *  - Calls that take a stream are ordered on it; when an output is a host
 *    scalar the call synchronises the stream before returning.  A NULL stream
 *    is the legacy default stream.
 *  - Vertices are 0..n-1; colours are 0..kc-1 (Sec. 2.3.1 draws colours in
 *    [0, k-1]).
 */
#ifndef SG2V_H
#define SG2V_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *sg2v_stream; /* a cudaStream_t */
typedef struct sg2v_graph sg2v_graph;
typedef struct sg2v_plan sg2v_plan;

typedef enum {
    SG2V_OK = 0,
    SG2V_ERR_INVALID_ARGUMENT = 1, /* null pointer, size out of range, bad flag */
    SG2V_ERR_NOT_A_TREE = 2,       /* parent array is not a tree, or root out of range */
    SG2V_ERR_COLOUR_OUT_OF_RANGE = 3,
    SG2V_ERR_GRAPH_NOT_SIMPLE = 4, /* self-loop, duplicate arc, unsorted row, asymmetric CSR or weights */
    SG2V_ERR_OUT_OF_MEMORY = 5,
    SG2V_ERR_FP_OVERFLOW = 6,      /* a count left the range of the table type (inf/NaN; 2^64 or 2^128 for integers) */
    SG2V_ERR_CUDA = 7,             /* a CUDA runtime call failed; see sg2v_last_error() */
    SG2V_ERR_TIMEOUT = 8,          /* a bounded device-side wait gave up */
    SG2V_ERR_UNSUPPORTED = 9       /* a valid request this build cannot run (e.g. integer tables on a weighted graph) */
} sg2v_status;

typedef enum {
    SG2V_FP64 = 0,       /* count tables and sums in FP64 */
    SG2V_FP32 = 1,       /* count tables in FP32, final reductions in FP64 */
    SG2V_FP32_SCALED = 2, /* FP32 tables whose rows carry a power-of-two exponent
                          * (int16): a row's values are its stored values times
                          * 2^E, its largest stored value lies in [1, 2), so
                          * counts far beyond FP32's 2^128 (k = 15 on large
                          * graphs) keep FP32 relative precision; entries below
                          * 2^-126 of their row's largest, after the gather's
                          * alignment to the row's largest neighbour exponent,
                          * are flushed to zero.  Forward counts only. */
    SG2V_U64 = 3,        /* count tables in unsigned 64-bit integers: every
                          * value of the DP on an unweighted graph is an integer
                          * (Alg. 3 / 5), so counts are exact while every table
                          * entry stays below 2^64, past FP64's 2^53; a sum or
                          * product that wraps is detected and the call returns
                          * SG2V_ERR_FP_OVERFLOW.  Unweighted graphs and forward
                          * counts only (SG2V_ERR_UNSUPPORTED otherwise). */
    SG2V_U128 = 4        /* as SG2V_U64 with unsigned 128-bit counts (two 64-bit
                          * words, 16 bytes per entry): exact to 2^128. */
} sg2v_precision;

/* ------------------------------------------------------------------ graph */

#define SG2V_GRAPH_SKIP_VALIDATION 0x1u /* trust the CSR (no simplicity/symmetry check) */
#define SG2V_GRAPH_KEEP_ORDER 0x2u      /* keep the caller's vertex order on the device */

/*
 * sg2v_graph_create -- the input network as a sparse adjacency matrix A_G in
 * CSR form (Sec. 5.1: A_G(i,j) = 1 iff V_j is a neighbour of V_i; Table 1).
 *
 *   n        number of vertices (>= 1, < 2^31)
 *   nnz      number of stored arcs = 2 * undirected edges (< 2^31)
 *   row_ptr  [n+1] int64, host or device; row_ptr[0] = 0, row_ptr[n] = nnz
 *   col_idx  [nnz] int32, host or device; strictly increasing within a row
 *   weights  [nnz] float32, host or device, or NULL for the 0-1 matrix; the
 *            weighted form uses A_G.val of Alg. 4 (each embedding then
 *            contributes the product of its edge weights); weights[e] must
 *            equal the weight of the reverse arc and be finite and >= 0
 *   flags    0 or a combination of SG2V_GRAPH_SKIP_VALIDATION and
 *            SG2V_GRAPH_KEEP_ORDER
 *   out      receives the handle
 *
 * The graph must be simple and undirected: the CSR must be symmetric, with no
 * self-loops and no repeated arcs (Sec. 2.2.1: simple graph); violations give
 * SG2V_ERR_GRAPH_NOT_SIMPLE unless validation is skipped.  The library copies
 * the arrays onto the current device (the caller may free its copies) and
 * derives its load-balanced work list there: rows longer than a chunk (the
 * environment variable SG2V_CHUNK, else 512 arcs when the average degree is
 * at most 64 and 1,024 above) become several tasks whose partial results fold
 * into the row; SG2V_PANELS > 1 also cuts the work list into that many column
 * panels (the CSC-Split form of Alg. 6).  Unless SG2V_GRAPH_KEEP_ORDER is
 * given, the device copy numbers the vertices by decreasing degree (the rows
 * most arcs gather share cache lines); this is invisible to the caller:
 * colourings, per-vertex counts, per-vertex gradient seeds, weights and
 * per-arc gradients are always in the caller's vertex and arc order.  In that
 * order the vertices without arcs come last, and forward counting runs no
 * work for them (their per-vertex counts are zero; a single-vertex template
 * counts them as usual).
 * Errors: INVALID_ARGUMENT, GRAPH_NOT_SIMPLE, OUT_OF_MEMORY, CUDA.
 */
sg2v_status sg2v_graph_create(int64_t n, int64_t nnz, const int64_t *row_ptr, const int32_t *col_idx,
                              const float *weights, uint32_t flags, sg2v_graph **out);

/* Frees the device copies.  NULL is accepted. */
sg2v_status sg2v_graph_destroy(sg2v_graph *graph);

/* n, nnz, the largest degree and whether the graph carries weights. */
sg2v_status sg2v_graph_info(const sg2v_graph *graph, int64_t *n, int64_t *nnz, int64_t *max_degree,
                            int32_t *weighted);

/* ------------------------------------------------------------------- plan */

/*
 * sg2v_template_plan -- partitions the template (Sec. 2.3.2, Alg. 5 line
 * "Partition T into sub-templates").  Pure host work; needs no GPU.
 *
 *   k           template vertices, 1 <= k <= 16
 *   parent      [k] int32, host: parent[i] is i's parent, exactly one -1
 *   root        rho in [0, k): the tree is re-rooted at rho (the per-vertex
 *               counts are "rho mapped to v")
 *   num_colours kc, k <= kc <= 16 (Sec. 2.3.1 takes kc = k)
 *   opts        NULL, or a sg2v_plan_opts (below)
 *   out         receives the handle
 *
 * Split rule: at a sub-template rooted at x, one edge (x, tau) to a kept
 * child is cut (Sec. 2.3.2 leaves the choice open); the part holding x is
 * the active child, the cut-off subtree (rooted at tau) the passive child.
 * SG2V_CUT_LAST (the default) cuts the edge to x's last remaining child
 * (children ordered by vertex index).  SG2V_CUT_MIN_WORK picks, at every
 * node, the child that minimises a model of the DP's work per vertex (the
 * gathered compressed rows times avg_degree, the eMA products, the output
 * writes; measured relative costs on B300), and keeps the default plan
 * unless the model, sharing counted, gains at least 1%.  The counts do not
 * depend on the choice.  Sub-templates that are isomorphic as rooted trees
 * share one table.
 * Errors: INVALID_ARGUMENT, NOT_A_TREE, UNSUPPORTED (kc > 16).
 */
#define SG2V_CUT_LAST 0
#define SG2V_CUT_MIN_WORK 1
typedef struct {
    uint32_t size;      /* sizeof(sg2v_plan_opts) */
    int32_t cut;        /* SG2V_CUT_LAST or SG2V_CUT_MIN_WORK */
    float avg_degree;   /* arcs per vertex of the graphs to count (0: 32) */
} sg2v_plan_opts;

sg2v_status sg2v_template_plan(int32_t k, const int32_t *parent, int32_t root, int32_t num_colours,
                               const void *opts, sg2v_plan **out);

sg2v_status sg2v_plan_destroy(sg2v_plan *plan);

/*
 * sg2v_plan_info -- alpha (automorphisms of the unrooted template, Alg. 1),
 * the number of DP nodes after sharing, and the widest table in columns
 * (C(kc, t) for the largest sub-template size t).  Any output may be NULL.
 */
sg2v_status sg2v_plan_info(const sg2v_plan *plan, int64_t *automorphisms, int32_t *num_nodes, int64_t *max_cols);

/*
 * sg2v_plan_nodes -- the DP nodes in execution order (children first).
 * out[6*i .. 6*i+5] = { t, a, p, active node or -1 (single vertex),
 *                       passive node or -1 (single vertex), is_root }.
 * capacity is the number of int32 entries available in out.
 */
sg2v_status sg2v_plan_nodes(const sg2v_plan *plan, int32_t *out, int64_t capacity);

/*
 * sg2v_plan_estimate_scale -- 1/(P * alpha) of Alg. 1 with
 * P = kc! / ((kc-k)! * kc^k), so that estimate = total * scale.
 */
sg2v_status sg2v_plan_estimate_scale(const sg2v_plan *plan, double *scale);

/* ------------------------------------------------------------------ count */

/*
 * sg2v_count -- one colouring through the whole DP (Alg. 5 inner loop:
 * SpMM + eMA per sub-template, then the root reduction and finalCount).
 *
 *   colours     [n] int8, host or device, values in [0, kc)
 *   precision   SG2V_FP64, SG2V_FP32, SG2V_FP32_SCALED, SG2V_U64 or
 *               SG2V_U128 (table type); an SG2V_FP32 call that overflows is
 *               run again as SG2V_FP32_SCALED by sg2v_count and
 *               sg2v_count_batched
 *   per_vertex  [n] double, host or device, or NULL: per_vertex[v] is the
 *               number of colourful embeddings (labelled maps) with the
 *               root rho at v, i.e. sum over colour sets C of M_0(v, I_C)
 *   total       host double or NULL: sum_v per_vertex[v]; FP64 counts are
 *               summed exactly in 128-bit integers when they are integral
 *   estimate    host double or NULL: total / (P * alpha)
 *   stream      CUDA stream
 *
 * Workspace (count tables) is allocated stream-ordered on the current device
 * and released before return.  Errors: INVALID_ARGUMENT,
 * COLOUR_OUT_OF_RANGE, OUT_OF_MEMORY, FP_OVERFLOW, UNSUPPORTED, CUDA.
 */
sg2v_status sg2v_count(const sg2v_graph *graph, const sg2v_plan *plan, const int8_t *colours,
                       sg2v_precision precision, double *per_vertex, double *total, double *estimate,
                       sg2v_stream stream);

/*
 * sg2v_count_batched -- B independent colourings for each of num_plans
 * templates in one pass: colourings become extra columns of every table row
 * (row v holds B consecutive colour-set blocks), so each CSR sweep serves
 * all B colourings, and sub-templates isomorphic across the plans share
 * tables.  All plans must use the same num_colours.
 *
 *   plans       [num_plans] plan handles
 *   colours     [B][n] int8, host or device
 *   per_vertex  [num_plans][B][n] double, host or device, or NULL
 *   totals      [num_plans][B] double, host or device, or NULL
 *   estimates   [num_plans][B] double, host or device, or NULL
 * Errors as sg2v_count.
 */
sg2v_status sg2v_count_batched(const sg2v_graph *graph, const sg2v_plan *const *plans, int32_t num_plans,
                               const int8_t *colours, int32_t B, sg2v_precision precision, double *per_vertex,
                               double *totals, double *estimates, sg2v_stream stream);

/* --------------------------------------------------------------- backward */

/*
 * sg2v_count_backward -- gradient of the weighted count with respect to the
 * edge weights (the differentiable form; the paper counts unweighted
 * graphs, Sec. 2.2.1, and Alg. 4's A_G.val carries the weights here).  For a
 * colouring, F(w) = sum_v g_v * per_vertex[v](w) where each colourful map
 * contributes the product of the weights of its k - 1 edges, so F is
 * multilinear in the weights.  The library runs the forward DP keeping every
 * table and every node's Y', then, parents before children, the reverse
 * eMA, the transposed SpMM (A symmetric) and a per-arc SDDMM
 * dF/dw_vu = <Ybar(v, .), M_p(u, .)>, and sums both arcs of each edge.
 *
 *   colours          [n] int8, host or device
 *   grad_per_vertex  [n] double (g_v), host or device, or NULL for g = 1
 *                    (the gradient of the total)
 *   grad_weights     [nnz] double, host or device: for every arc, dF/dw_e of
 *                    its undirected edge e (both arcs of an edge hold the
 *                    same value); unweighted graphs give the derivative at
 *                    w = 1 (the colourful maps through each edge)
 *   total            host double or NULL: the forward total sum_v per_vertex[v]
 *   flags            0 (choose the form by memory), SG2V_BACKWARD_STORE or
 *                    SG2V_BACKWARD_RECOMPUTE (not both)
 * Memory: the stored form keeps every node's table, Y' and gradient table
 * of the colouring during the call.  The recompute form keeps only what the
 * current reverse step reads: the tables of the node's children are rebuilt
 * by replaying the forward of their sub-templates (the storage discipline of
 * Sec. 5.3 / Alg. 5 applied to the reverse walk), the node's Y' by replaying
 * its gather, and all of it is freed after the step; it costs more launches
 * and gives the same gradients (bit for bit when no row is split into
 * chunks: the same kernels produce each value; split rows fold their chunks
 * with atomic adds, whose order can change the last bits).  With flags = 0
 * the stored form is used
 * when it fits 80% of the device's free memory, else the recompute form.
 * sg2v_last_call_peak_bytes reports the call's peak workspace.  Errors as
 * sg2v_count; SG2V_FP32_SCALED is UNSUPPORTED here.
 */
#define SG2V_BACKWARD_RECOMPUTE 0x1u
#define SG2V_BACKWARD_STORE 0x2u
sg2v_status sg2v_count_backward(const sg2v_graph *graph, const sg2v_plan *plan, const int8_t *colours,
                                sg2v_precision precision, const double *grad_per_vertex, double *grad_weights,
                                double *total, uint32_t flags, sg2v_stream stream);

/*
 * sg2v_graph_set_weights -- replaces the weights of a graph created with
 * weights ([nnz] float32, host or device, stream-ordered copy).  No
 * validation: weights[e] must equal the reverse arc's weight and be finite
 * and >= 0.  Used by the autograd wrapper between iterations.
 */
sg2v_status sg2v_graph_set_weights(sg2v_graph *graph, const float *weights, sg2v_stream stream);

/* ---------------------------------------------------------------- session */

/*
 * A session runs the same request (graph, plans, B colourings, precision)
 * many times with new colourings, asynchronously and without allocating:
 * every buffer is allocated once at creation, the whole launch sequence of a
 * run (colour check, per wave the colour sort and one launch per DP node,
 * root reductions and the final totals) is captured into a CUDA graph on the
 * first run and replayed afterwards, and totals and estimates are finished on
 * the device (exact 128-bit sums rounded once; estimates in double-double).
 * This is the batched form of the method for repeated colourings (the
 * estimator of Alg. 1 runs N colourings).  Not thread-safe: one run at a time
 * per session.
 */
typedef struct sg2v_session sg2v_session;

#define SG2V_SESSION_PER_VERTEX 0x1u /* keep per-vertex counts ([plans][B][n] doubles) */
#define SG2V_SESSION_NO_GRAPH 0x2u   /* launch kernels directly instead of replaying a CUDA graph */
#define SG2V_SESSION_AUTOTUNE 0x4u   /* the first run times candidate wave widths and node forms (below) */

/*
 * sg2v_session_create -- plans as in sg2v_count_batched (same num_colours),
 * B >= 1 colourings per run, flags from SG2V_SESSION_*.  Device memory of
 * the current device is allocated here (OUT_OF_MEMORY if it does not fit).
 */
sg2v_status sg2v_session_create(const sg2v_graph *graph, const sg2v_plan *const *plans, int32_t num_plans,
                                int32_t B, sg2v_precision precision, uint32_t flags, sg2v_session **out);

/*
 * sg2v_session_run -- one run on stream.  colours [B][n] int8, host or
 * device, is copied into the session first; totals / estimates
 * ([num_plans][B] doubles) and per_vertex ([num_plans][B][n], requires
 * SG2V_SESSION_PER_VERTEX) may be NULL, host or device and are written by
 * copies ordered after the run.  Returns without synchronising (except the
 * first run of an autotuning session, which times candidates); errors found
 * by the kernels (colour range, overflow) are reported by sg2v_session_sync.
 */
sg2v_status sg2v_session_run(sg2v_session *session, const int8_t *colours, double *totals, double *estimates,
                             double *per_vertex, sg2v_stream stream);

/* Waits for the session's last run on stream and returns its status
 * (COLOUR_OUT_OF_RANGE, FP_OVERFLOW or OK). */
sg2v_status sg2v_session_sync(sg2v_session *session, sg2v_stream stream);

/* Wave width in use (colourings sharing a table row) and whether runs replay
 * a CUDA graph.  Either output may be NULL. */
sg2v_status sg2v_session_info(const sg2v_session *session, int32_t *wave, int32_t *graph);

/*
 * Autotuning (SG2V_SESSION_AUTOTUNE).  The first run times, in this order,
 * the split schedule: the chunk size (256 to 8192 arcs, up to the first size
 * that splits no row) at which rows longer than it are cut into tasks whose
 * partial results fold into the row, then, at the best size, work lists in
 * 2 and 4 column panels (rows also cut where their neighbours cross into the
 * next range of vertices, tasks run panel by panel: the CSC-Split form of
 * Alg. 6); the whole step is timed on each candidate's work list.  The
 * environment variables SG2V_CHUNK and SG2V_PANELS, read at graph creation,
 * fix either instead.  It then times the candidate
 * wave widths and, at the chosen width, the forms each DP node can take:
 * the run-scatter kernel or per-colour accumulators, short narrow rows one
 * per lane group or one per warp, histogram nodes 32 rows per warp or one,
 * a large eMA in its own launch or in the gather's epilogue.  Each node
 * keeps its fastest form (per-node CUDA-event times; results do not depend
 * on the form).  When the environment variable SG2V_TUNE_CACHE names a file,
 * the choices are stored there as JSON, keyed by graph statistics (vertices,
 * arcs, largest degree, weights), colours, node shape, table type, wave and
 * chunk size (the split schedule by the graph statistics, colours, table
 * type, colourings and templates), and a later session finding its keys in
 * the file takes them without timing them again (the wave width is always
 * timed).
 *
 * sg2v_session_tuning -- the session's choices as JSON text
 * ({"wave": W, "chunk": C, "panels": P, "tuned": bool, "nodes": [{"t", "a", "p", "kernel",
 * "lane_groups", "deferred_ema", "form"}, ...]}), NUL-terminated in out
 * (capacity bytes, truncated if short); *length (may be NULL) gets the full
 * length without the NUL.
 */
sg2v_status sg2v_session_tuning(const sg2v_session *session, char *out, int64_t capacity, int64_t *length);

sg2v_status sg2v_session_destroy(sg2v_session *session);

/* -------------------------------------------------------------- profiling */

/*
 * Kernel timing (not part of the paper's method; measurement support).
 * While enabled, every count call records a CUDA event pair on its stream
 * around each kernel it launches and, after its final synchronisation, adds
 * the elapsed times to a per-kernel record keyed by the kernel's role
 * ("node t=10 a=5 p=5 fp32", "root_reduce", ...).  Records also carry the
 * kernel's algorithmic bytes (each input table, CSR array and colouring read
 * once, each output written once) so that callers can report achieved
 * bandwidth.  The records are process-wide and guarded by a mutex.
 */
typedef struct {
    char name[64];
    int64_t launches;
    double total_ms;        /* sum of event-timed durations */
    double bytes_per_launch; /* algorithmic bytes of one launch */
} sg2v_kernel_record;

sg2v_status sg2v_profile_enable(int32_t enable);
sg2v_status sg2v_profile_reset(void);
/* Copies up to capacity records into out and their number into *count. */
sg2v_status sg2v_profile_read(sg2v_kernel_record *out, int32_t capacity, int32_t *count);
/* Kernels launched by count calls since the last reset (profiling or not). */
int64_t sg2v_launch_count(void);

/* ------------------------------------------------------- allocation-free */

/*
 * sg2v_sum_counts_noalloc -- sums per-vertex counts into totals without
 * allocating anything.  The paper has no counterpart; this is a service for
 * callers that cannot allocate device memory where they need a total:
 * serving loops whose device memory is reserved up front by their own
 * allocator (where a further allocation may fail or be forbidden), and code
 * that must not stall other streams (cudaMalloc and cudaFree synchronise the
 * device).
 *
 *   values  [nseg][n] double, device memory: e.g. the per_vertex output of
 *           sg2v_count / sg2v_count_batched
 *   n       values per segment, >= 1
 *   nseg    segments, 1 <= nseg <= 1024 (larger requests are rejected with
 *           SG2V_ERR_INVALID_ARGUMENT and nothing is launched)
 *   totals  [nseg] double, device memory: totals[s] = sum of segment s.  When
 *           every value is a non-negative integer below 2^128 the sum is
 *           exact and rounded once to the nearest double (the same value
 *           sg2v_count reports); otherwise it is a compensated FP64 sum; a
 *           non-finite value gives a non-finite total
 *   stream  the call is stream-ordered and returns without synchronising
 *
 * Scratch: a fixed 2.5 MiB device array inside the library (one partial sum
 * per segment and block), which every GPU that loads the library keeps until
 * the process exits.  The first call on a device looks up that array's
 * device address (cudaGetSymbolAddress) with the device current; make that
 * first call before any stream capture.  Each call overwrites the records it
 * reads, so nothing carries over between calls, but all calls share the
 * array: calls whose kernels overlap on the GPU (different streams without
 * ordering) race and give wrong totals.  The looked-up address is kept for
 * the life of the process: do not call this entry point on a device after
 * cudaDeviceReset on it.
 * Errors: INVALID_ARGUMENT (null, sizes, host pointers), CUDA.
 */
sg2v_status sg2v_sum_counts_noalloc(const double *values, int64_t n, int32_t nseg, double *totals,
                                    sg2v_stream stream);

/* -------------------------------------------------------------- allocator */

/*
 * sg2v_set_allocator -- where per-call device workspaces come from.  The
 * paper has no counterpart (its CPU code allocates its tables itself); the
 * hook lets a caller that manages device memory (e.g. PyTorch's caching
 * allocator) serve the library's temporary buffers.
 *
 *   alloc  alloc(bytes, stream, user) returns device memory of at least
 *          `bytes` usable in stream order on `stream`, 16-byte aligned, or
 *          NULL when it has none (the call then fails with
 *          SG2V_ERR_OUT_OF_MEMORY after returning what it already took)
 *   free   free(ptr, stream, user) takes back a block of alloc; the library
 *          calls it in stream order after the block's last use on `stream`
 *   user   passed through
 *
 * Both NULL restores the default: the library's stream-ordered pool of the
 * current device.  Covered: the per-call buffers of sg2v_count,
 * sg2v_count_batched and sg2v_count_backward (colour-sorted arcs, tables,
 * scratch), and the buffers of sessions created while the hook is set (taken
 * at sg2v_session_create on the default stream, given back at
 * sg2v_session_destroy after a device synchronisation; a session keeps the
 * hook it was created with, so alloc, free and user must stay valid until
 * every such session is destroyed).  Graph and plan handles are not covered (they
 * live until their destroy call).  The setting is process-wide: change it
 * only while no call is running.  Errors: INVALID_ARGUMENT (exactly one of
 * alloc / free given).
 */
typedef void *(*sg2v_alloc_fn)(size_t bytes, sg2v_stream stream, void *user);
typedef void (*sg2v_free_fn)(void *ptr, sg2v_stream stream, void *user);
sg2v_status sg2v_set_allocator(sg2v_alloc_fn alloc, sg2v_free_fn free, void *user);

/*
 * sg2v_last_call_peak_bytes -- the largest amount of per-call device
 * workspace (tables, sorted arcs, scratch) that the last sg2v_count,
 * sg2v_count_batched or sg2v_count_backward call of the calling thread held
 * at once, in bytes (0 before any call).  Graph, plan and session memory is
 * not included.
 */
int64_t sg2v_last_call_peak_bytes(void);

/* ---------------------------------------------------------------- status */

/* Static English name of a status code. */
const char *sg2v_status_string(sg2v_status status);

/* Detail of the last failure on the calling thread ("" if none). */
const char *sg2v_last_error(void);

/* Library version as major*10000 + minor*100 + patch. */
int32_t sg2v_version(void);

#ifdef __cplusplus
}
#endif

#endif /* SG2V_H */
