// Device kernels of the colour-coding DP and their launchers.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

namespace sg2v {

// Element type of the count tables: FP32, FP64, or unsigned 64-bit or
// 128-bit integers (exact counts; every wrap past 2^64 / 2^128 is reported).
enum class Elem : int { F32 = 0, F64 = 1, U64 = 2, U128 = 3 };

// Arguments of one DP node over a batch of nb colourings.  Tables are
// colour-compressed: row v*nb + b holds, for colouring b of vertex v, only the
// colour sets containing v's colour, indexed by the colex rank of the other
// colours in the squeezed universe (kc - 1 colours), with `ld*` elements
// between rows (ld is a multiple of 16 bytes).
struct NodeArgs {
    // graph (CSR) and the load-balanced work list
    const int64_t *row_ptr;
    const int32_t *col_idx;
    const float *weights;         // per-arc weights, or null
    const int4 *tasks;            // {row, split slot or -1, first arc, end arc} (arc indices into col_idx)
    int64_t ntasks;
    const int32_t *heavy_chunks;  // tasks per split slot
    int64_t n;
    int nb;                       // colourings in the batch
    const int8_t *colours;        // [nb][n]
    int kc;
    // arcs of every row sorted by neighbour colour, per colouring: [nb][nnz]
    // (neighbour, its colour or -1 when outside [0, kc), weight)
    int64_t nnz;
    const int32_t *scol;
    const int8_t *sclr;
    const float *sw;              // null when unweighted
    // passive side: per-colour accumulators Z(d, i) of compressed rows of
    // width Wz = C(kc-1, p-1), or the colour histogram when hist != 0
    const void *Mp;
    int64_t ldp;
    int Wz;
    int wz_pad;                   // Z row stride in elements: narrow rows (lane groups) the row's
                                  // 16-byte vectors, warp- and CTA-wide rows their lanes' whole tile
    int hist;
    // Y' (p-sets without v's colour) from Z
    int p;
    int wy;                       // C(kc-1, p)
    const uint16_t *expand;       // [kc][wy][pstride] offsets into Z (the first p of each set)
    const uint32_t *expand32;     // [kc][wy][p] 32-bit offsets instead (Z of more than 65,536
                                  // elements: CTA-wide rows only), else null
    int pstride;                  // p, 4 when 2 <= p <= 4, 8 when 5 <= p <= 8 (8-byte loads)
    // histogram nodes: neighbour counts per colour written by the colour sort
    // ([n * nb][hld] int32, the full row's counts even for split rows), or null
    const int32_t *hcount;
    int hld;
    // shared memory per warp, in elements: Z copies, Y', the active row
    int zwords, ywords, mwords;
    // active side
    const void *Ma;
    int64_t lda;
    int Wa;                       // C(kc-1, a-1)
    int a_leaf;                   // active child is a single vertex: M_s' = Y'
    // output
    void *Ms;
    int64_t ldt;
    int Ws;                       // C(kc-1, t-1)
    int root;                     // sum the row of M_s' into root_out instead of storing it
    void *root_out;               // [nb][n]
    const uint32_t *splits;       // [Ws][nsplit] rank(A') | rank(S' - A') << 16 (a >= 2)
    int nsplit;
    // root with t = kc (one output set S', so each p-set P' of Y' pairs with
    // exactly one A' = S' - P'): rootpair[rank(P')] = rank(A'), [wy], wy <= 128;
    // null otherwise.  The row sum is then sum over P' of M_a'(A') * Y'(P').
    const uint16_t *rootpair;
    // FP32 range: per-row power-of-two exponents (scaled != 0).  A row's true
    // values are its stored values times 2^E[row]; Eref[row] is the largest
    // exponent among the neighbours the row gathers (colour != own colour).
    int scaled;
    const int16_t *Ep;            // exponents of the passive table rows (p >= 2)
    const int16_t *Ea;            // exponents of the active table rows (a >= 2)
    int16_t *Es;                  // exponents of the output rows (non-root)
    const int32_t *Eref;          // [n * nb]
    double *root_out_d;           // root per-vertex values (scaled): [nb][n]
    int owords;                   // shared-memory words per warp (or CTA) for the output row (scaled)
    // backward support: also store Y' rows (Yout != null); add the output row
    // to the existing one instead of overwriting it (accumulate != 0)
    void *Yout;
    int64_t ldy;
    int accumulate;
    // root whose active and passive children are one table, totals only: the
    // contribution of an arc (v, u) to v's count equals that of (u, v) to u's,
    // so only arcs with u < v are gathered and the row sum is doubled (the
    // per-vertex values are then not the per-vertex counts); with vertices
    // numbered by decreasing degree the gathered row is the edge's hub end,
    // the one most likely in L2
    int half_arcs;
    // large eMA: the gather kernel stores Y' rows in Yout (ldy) and skips the
    // eMA, which launch_ema_rows then runs over blocks of rows
    int defer;
    // narrow rows: each group of lanes (lanes_per_group) takes its own task
    // (node_group_kernel); shared memory per warp is then
    // (32 / lanes) * (kc * wz_pad + ywords + mwords + owords) elements
    int group_rows;
    // CTA-wide rows: column tiles walked per row (npass >= 1), and Z in
    // global memory ([grid][kc][wz_pad], this CTA's slot at blockIdx.x) when
    // it does not fit shared memory (null: Z in shared memory)
    int npass;
    void *zglobal;
    // FP32 gathers: lanes past the row's last 16-byte vector load nothing
    // (else they read the next row into Z columns nothing reads)
    int pred_lanes;
    // run-scatter kernel: for the row's colour cv and a neighbour colour d,
    // runmap[(cv * kc + d) * wmap + e] is where entry e of a gathered row
    // goes: a Y' index (a sink index past Y' when the entry's set holds cv)
    // or, at a root with one output set, the index of the active-row entry it
    // pairs with (mzero, a zero, when the set holds cv)
    const uint16_t *runmap;
    int wmap;
    int mzero;
    // run-scatter kernel: 16-byte vectors between consecutive vertex rows of
    // the passive table (nb * ldp / entries per vector; set by its launcher)
    unsigned uvec;
    // rows [live_rows, n) belong to isolated vertices whose tasks do not run
    // (their table rows are never read); n when every row runs
    int64_t live_rows;
    // run-scatter kernel: data read or written once per launch (sorted arcs,
    // active rows, output rows) carry an L2 evict-first hint (l2_stream != 0),
    // so the gathered table keeps more of L2
    int l2_stream;
    // partial Z of split (heavy) rows
    void *scratch;                // [slots][nb][scratch_ld]
    int64_t scratch_ld;
    unsigned *counters;           // [slots][nb], zero on entry
    // status word 0 of the call: integer tables set bit 1 when a count
    // wrapped past their width
    unsigned *status;
};

// Backward of the eMA of one node for one colouring (one warp per row):
//   Ybar'(P') = sum over S' containing P' of G'(S') * M_a'(S' - P')
//   Gabar'(A') += sum over S' containing A' of G'(S') * Y'(S' - A')
// (a = 1: Ybar' = G').  At the root G'(S') is the per-vertex seed.
struct BwdEmaArgs {
    int64_t n;
    const int8_t *colours;
    int kc, a;
    int ws, wa, wy;               // C(kc-1, t-1), C(kc-1, a-1), C(kc-1, p)
    const void *G;                // [n][ldg] gradient of M_s' (null at the root)
    int64_t ldg;
    const double *seed;           // [n] gradient of the per-vertex counts (root)
    const void *Ma;
    int64_t lda;
    const void *Y;
    int64_t ldy;
    void *Ybar;                   // out [n][ldyb]
    int64_t ldyb;
    void *Gabar;                  // accumulated [n][ldga] (a >= 2)
    int64_t ldga;
    const uint32_t *ybar;         // [wy][nybar]
    int nybar;
    const uint32_t *mabar;        // [wa][nmabar]
    int nmabar;
};

// Per-arc weight gradient of one node (one warp per row u, arcs in CSR
// order): grad[e] += sum over the arc table of Ybar'(v, .) * M_p'(u, .) for
// arc e = (u, v); M_p' = 1 when the passive child is a single vertex.
struct SddmmArgs {
    int64_t n;
    const int64_t *row_ptr;
    const int32_t *col_idx;
    const int8_t *colours;
    int kc, hist;
    const void *Ybar;
    int64_t ldyb;
    const void *Mp;
    int64_t ldp;
    int wmp;                      // C(kc-1, p-1)
    const uint32_t *arc;          // [kc][kc][narc]
    int narc;
    double *grad;                 // [nnz]
    // the work list of the forward pass (null: one warp per row), and for the
    // row-oriented form (p >= 2, lanes > 0) the gather shape of rows of wmp
    // elements (lanes per group, vectors per lane)
    const int4 *tasks;
    int64_t ntasks;
    int lanes, vecs, wz_pad;
    // sorted form (row form with scol != null): the forward's colour-sorted
    // arcs of every task with each one's arc index (perm), and the node's run
    // map ([kc][kc][wmap]: for v's colour and the neighbour's colour, where
    // entry e of the neighbour's row sits in v's Ybar' row, or ysink, a zero)
    const int32_t *scol;
    const int8_t *sclr;
    const int32_t *perm;
    const uint16_t *runmap;
    int wmap, ysink, ywords;
};

cudaError_t launch_bwd_ema(const BwdEmaArgs &args, bool fp64, int sms, cudaStream_t stream);
cudaError_t launch_sddmm(const SddmmArgs &args, bool fp64, int sms, cudaStream_t stream);
// whether the sorted form of the per-arc gradient exists for this row shape
bool sddmm_sorted_available(bool fp64, int lanes, int vecs);
// grad_w[arcmap[e]] = part[e] + part[rev[e]] (arcmap null: grad_w[e])
cudaError_t launch_symmetrize(const double *part, const int32_t *rev, const int32_t *arcmap, int64_t nnz,
                              double *grad_w, cudaStream_t stream);
// dst[b * n + i] = src[b * n + idx[i]] (colourings into the graph's vertex
// order, weights into its arc order, per-vertex seeds)
cudaError_t launch_gather_i8(const int8_t *src, int8_t *dst, const int32_t *idx, int64_t n, int nb,
                             cudaStream_t stream);
cudaError_t launch_gather_f32(const float *src, float *dst, const int32_t *idx, int64_t n, cudaStream_t stream);
cudaError_t launch_gather_f64(const double *src, double *dst, const int32_t *idx, int64_t n, cudaStream_t stream);

// Per-segment (template x colouring) result of the root reduction.
struct RootSum {
    unsigned long long lo, hi;    // exact 128-bit integer sum (valid when flags == 0)
    double s, c;                  // compensated FP64 sum s + c
    unsigned flags;               // bit 0: a value was not an integer; bit 1: non-finite value
    unsigned pad;
};

// Exponent of a table row whose entries are all zero (scaled FP32).
constexpr int kEmptyRowExp = -32768;

constexpr unsigned kFlagNotIntegral = 1u;
constexpr unsigned kFlagNonFinite = 2u;

// Resident blocks per SM / launch of the scaled FP32 variants (per-row exponents).
int node_blocks_per_sm_scaled(bool hist, int lanes_per_group, int vec_per_lane, bool weighted, int threads,
                              size_t smem, bool group_rows = false);
cudaError_t launch_node_scaled(const NodeArgs &args, int lanes_per_group, int vec_per_lane, int threads, size_t smem,
                               int grid_cap, cudaStream_t stream);

// Shape of the gather of compressed rows of wz elements: lanes per neighbour
// group (4, 8, 16 or 32; kWideLanes when a whole CTA shares one row) and
// 16-byte vectors per lane (1..4; 0 if too wide).
void node_shape(int elems_per_vector, int wz, int *lanes_per_group, int *vec_per_lane);

constexpr int kNodeThreads = 256;
// node_shape's lanes-per-group value for rows handled by a whole CTA (wide rows)
constexpr int kWideLanes = 256;
constexpr int kWideThreads = 256;

// Resident blocks per SM of one node-kernel variant at a block size and
// dynamic shared-memory size (0 if it cannot run); raises the kernel's
// shared-memory limit when needed.
int node_blocks_per_sm(Elem e, bool hist, int lanes_per_group, int vec_per_lane, bool weighted, int threads,
                       size_t smem, bool group_rows = false);

// Run-scatter node kernel (run_kernel.cu; plain FP32 tables, FP64 without
// weights): one task per warp, lane groups of g (4, 8, 16 or 32) covering a
// gathered row of g * nv vectors (nv = 2 only with g = 32); form 0 generic
// eMA epilogue, 1 single-vertex active child (M_s' = Y'), 2 root with one
// output set (row sum of pairs).  Shared memory per warp: (ywords + mwords)
// elements plus kRunCompactBytes.  0 blocks per SM when the variant does not
// exist.
constexpr int kRunCompactBytes = 384;
int node_run_blocks_per_sm(Elem e, int g, int nv, bool weighted, int form, int threads, size_t smem);
cudaError_t launch_node_run(const NodeArgs &args, Elem e, int g, int nv, int form, int threads, size_t smem,
                            int grid_cap, cudaStream_t stream);

// Launch helpers shared by the kernel files: resident blocks per SM of a
// kernel at a block size and dynamic shared memory (raising the kernel's
// shared-memory limit when needed; 0 if it cannot run), the same check made
// once per kernel at launch, and a node launch over the work list (grid
// capped at grid_cap; g lanes per task group, kWideLanes for one CTA per task).
int blocks_per_sm(void *kernel, int threads, size_t smem);
cudaError_t ensure_smem(void *kernel, int threads, size_t smem);
cudaError_t launch_variant(void *kernel, const NodeArgs &args, int g, int threads, size_t smem, int grid_cap,
                           cudaStream_t stream);

// Launches the fused SpMM/histogram + eMA kernel of one node.
cudaError_t launch_node(const NodeArgs &args, Elem e, int lanes_per_group, int vec_per_lane, int threads,
                        size_t smem, int grid_cap, cudaStream_t stream);

// Deferred eMA of a non-root node (a >= 2) over blocks of kEmaRows rows: Y'
// rows from Yout (written by the node's gather launch with defer set), the
// active rows from Ma, outputs (and, scaled, exponents) to Ms / Es.  Each
// split-table word serves kEmaRows rows.  0 blocks per SM if the rows of a
// block do not fit shared memory.
constexpr int kEmaRows = 8;
size_t ema_rows_smem(const NodeArgs &args, Elem e, bool scaled);
int ema_rows_blocks_per_sm(Elem e, bool scaled, size_t smem);
cudaError_t launch_ema_rows(const NodeArgs &args, Elem e, bool scaled, int sms, cudaStream_t stream);

// Histogram nodes in blocks of 32 rows per warp (counts with one lane per
// row, then the eMA epilogue row by row).  Shared memory per warp:
// (kc * 32 + 32 * mwords + ywords + owords) elements.
int hist_rows_blocks_per_sm(Elem e, bool scaled, bool weighted, int threads, size_t smem);
cudaError_t launch_hist_rows(const NodeArgs &args, Elem e, bool scaled, int threads, size_t smem, int grid_cap,
                             cudaStream_t stream);

// Root reduction: vals is [nseg][n] of float, double or unsigned 64-bit
// counts, of which entries [live, n) of each segment are zeros that are not
// read; writes per-vertex doubles when pv != null (value of vertex i at
// pv[seg * n + pvmap[i]], or at i when pvmap is null) and one RootSum per
// segment.
cudaError_t launch_root_reduce(const void *vals, Elem e, int64_t n, int64_t live, int nseg, double *pv,
                               const int32_t *pvmap,
                               RootSum *partials, int chunks, RootSum *out, cudaStream_t stream);

// Eref[row] = max over the row's arcs to neighbours of another valid colour
// of Ep[neighbour row] (Eref pre-filled below kEmptyRowExp, e.g. bytes 0x80; split rows combine
// chunks with atomicMax).
cudaError_t launch_eref(const int4 *tasks, int64_t ntasks, const int32_t *scol, const int8_t *sclr,
                        const int8_t *colours, int64_t n, int64_t nnz, int nb, int kc, const int16_t *Ep,
                        int32_t *Eref, int sms, cudaStream_t stream);

// Sorts the arcs of every work-list task by neighbour colour (stable) for
// each of nb colourings: scol/sclr/sw [nb][nnz] (sw only when weights != null).
// Tasks from small_begin on have at most kSortSmallArcs arcs (the work list
// is sorted by work) and sort several per warp.
constexpr int kSortSmallArcs = 8;
// The table of a histogram node whose children are both single vertices
// (t = 2), written by the sort from its bucket counts: row v * nb + b gets,
// for each colour x != col(v) in squeezed order, the number of v's
// neighbours of colour x (a row of zeros when col(v) is invalid).  Chunks of
// split rows add their counts atomically, so the table must be zero on entry
// when the graph has split rows.  out == null: no histogram.
struct SortHist {
    void *out;
    int64_t ld;                   // elements between rows
    Elem elem;
    // per-row neighbour counts of every colour for the other histogram nodes:
    // row v * nb + b holds hld int32 (entry c: neighbours of colour c, c < kc;
    // split rows add atomically into a zeroed buffer); null: none
    int32_t *hcount;
    int hld;
    // the arc index (into col_idx) of every sorted arc ([nb][nnz],
    // sorted positions), or null: maps per-arc results back to arc order
    int32_t *perm;
};
// The (2, 1, 1) table of a weighted graph (FP32 or FP64 tables) from the
// colour-sorted arcs: out[(v * nb + b) * ld + j] = the weights of v's arcs to
// the j-th colour other than col(v), summed; rows of split tasks must be zero.
// out2 (stride ld2, or null) receives the same rows: the node's Y'.  Tasks
// from small_begin on have at most kSortSmallArcs arcs (run 4 per warp).
cudaError_t launch_weighted_hist(const int4 *tasks, int64_t ntasks, int64_t small_begin, const int8_t *sclr,
                                 const float *sw, int64_t nnz, const int8_t *colours, int64_t n, int nb, int kc,
                                 void *out, int64_t ld, void *out2, int64_t ld2, Elem e, int sms,
                                 cudaStream_t stream);
cudaError_t launch_colour_sort(const int4 *tasks, int64_t ntasks, int64_t small_begin, const int32_t *col_idx,
                               const float *weights, int64_t n, int64_t nnz, const int8_t *colours, int nb, int kc,
                               int32_t *scol, int8_t *sclr, float *sw, const SortHist &hist, int sms,
                               cudaStream_t stream);

// Totals and estimates of nseg segments from their root sums: the exact
// 128-bit sum rounded once to double when every value was an integer, else
// the compensated sum; estimate = total * (scale_hi + scale_lo)[segment / nb]
// in double-double.  Non-finite sums set bit 1 of *status.
cudaError_t launch_finalize(const RootSum *sums, int nseg, int nb, const double *scale_hi, const double *scale_lo,
                            double *totals, double *estimates, unsigned *status, cudaStream_t stream);

// Sets *status |= 1 when any of count colours is outside [0, kc).
cudaError_t launch_check_colours(const int8_t *colours, int64_t count, int kc, unsigned *status,
                                 cudaStream_t stream);

}  // namespace sg2v
