// Device kernels of the colour-coding DP and their launchers.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

namespace sg2v {

// Arguments of one DP node over a batch of nb colourings.  Table rows are
// (vertex, colouring) pairs: row v*nb + b holds colouring b of vertex v, with
// `ld*` elements between rows (ld is a multiple of 16 bytes).
struct NodeArgs {
    // graph (CSR) and the load-balanced work list
    const int64_t *row_ptr;
    const int32_t *col_idx;
    const float *weights;         // per-arc weights, or null
    const int4 *tasks;            // {row, heavy slot or -1, first arc offset, end arc offset}
    int64_t ntasks;
    const int32_t *heavy_chunks;  // tasks per heavy slot
    int64_t n;
    int nb;                       // colourings in the batch
    const int8_t *colours;        // [nb][n]
    int kc;
    // passive side: Y = A * M_p (or the colour histogram when hist != 0)
    const void *Mp;
    int64_t ldp;
    int Wp;                       // columns of Y per colouring
    int hist;
    // active side
    const void *Ma;
    int64_t lda;
    int a_leaf;                   // active child is a single vertex: masked gather
    // output
    void *Ms;
    int64_t ldt;
    int Wt;                       // columns of M_s per colouring
    int root;                     // sum the row of M_s into root_out instead of storing it
    void *root_out;               // [nb][n]
    const int32_t *gather;        // [kc][Wt] (a_leaf)
    const uint32_t *splits;       // [Wt][nsplit] rank(S_a) | rank(S - S_a) << 16
    int nsplit;
    // partial sums of split (heavy) rows
    void *scratch;                // [slots][nb][scratch_ld]
    int64_t scratch_ld;
    unsigned *counters;           // [slots][nb], zero on entry
};

// Per-segment (template x colouring) result of the root reduction.
struct RootSum {
    unsigned long long lo, hi;    // exact 128-bit integer sum (valid when flags == 0)
    double s, c;                  // compensated FP64 sum s + c
    unsigned flags;               // bit 0: a value was not an integer; bit 1: non-finite value
    unsigned pad;
};

constexpr unsigned kFlagNotIntegral = 1u;
constexpr unsigned kFlagNonFinite = 2u;

// Launches the fused SpMM/histogram + eMA kernel of one node.  vec_per_lane
// (1..4) is the number of 16-byte vectors of Y each lane accumulates.
cudaError_t launch_node(const NodeArgs &args, bool fp64, int vec_per_lane, int grid_cap, cudaStream_t stream);

// Maximum resident blocks per SM of one node-kernel variant (for grid sizing).
int node_blocks_per_sm(bool fp64, bool hist, int vec_per_lane, bool weighted);

constexpr int kNodeThreads = 256;

// Shared memory of the node kernel for a given variant.
size_t node_smem_bytes(bool fp64, bool hist, int vec_per_lane);

// Root reduction: vals is [nseg][n] of float/double; writes per-vertex doubles
// when pv != null and one RootSum per segment.
cudaError_t launch_root_reduce(const void *vals, bool fp64, int64_t n, int nseg, double *pv, RootSum *partials,
                               int chunks, RootSum *out, cudaStream_t stream);

// Sets *status |= 1 when any of count colours is outside [0, kc).
cudaError_t launch_check_colours(const int8_t *colours, int64_t count, int kc, unsigned *status,
                                 cudaStream_t stream);

}  // namespace sg2v
