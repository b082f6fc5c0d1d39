// Device kernels of the decoupled colour-coding DP (SubGraph2Vec, Alg. 3 / 5).
//
// One launch per DP node s = (T_s, T_a, T_p) computes, for every vertex v and
// colouring b of the batch,
//   Y(v, P)  = sum over arcs (v, u) of w_vu * M_p(u, P)       (Alg. 4: SpMV,
//              batched over the C(kc, p) columns P as an SpMM, Alg. 6)
//   M_s(v,S) = sum over S_a in S with |S_a| = a of M_a(v, S_a) * Y(v, S - S_a)
//                                                             (Alg. 5: eMA)
// without writing Y to memory: a warp owns one (row, colouring) pair, keeps
// the row of Y in registers while it walks the row's arcs, stages it in
// shared memory and applies the eMA in the epilogue.  When the passive child
// is a single vertex, Y is the per-colour neighbour histogram (M_p(u, {c}) is
// 1 exactly when u has colour c); when the active child is a single vertex,
// M_a(v, {c}) is 1 exactly when v has colour c and the eMA becomes a masked
// gather M_s(v, S) = [col(v) in S] * Y(v, S - {col(v)}).
//
// Load balance for power-law degrees: rows longer than a chunk are cut into
// chunks (separate tasks); each chunk adds its partial Y to a scratch row
// with atomics and the last chunk to finish (an atomic counter) runs the
// epilogue.  Tasks are ordered by decreasing work and dealt round-robin to
// the warps of a grid sized to the resident capacity of the GPU.
#include <cuda_runtime.h>

#include <cstdint>

#include "kernels.cuh"

namespace sg2v {

namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kMaxHistColours = 16;

template <typename T>
struct Vec16;
template <>
struct Vec16<float> {
    using type = float4;
    static constexpr int n = 4;
    __device__ static float4 zero() { return make_float4(0.f, 0.f, 0.f, 0.f); }
    __device__ static void add(float4 &a, const float4 &b) {
        a.x += b.x;
        a.y += b.y;
        a.z += b.z;
        a.w += b.w;
    }
    __device__ static void fma(float4 &a, float w, const float4 &b) {
        a.x = fmaf(w, b.x, a.x);
        a.y = fmaf(w, b.y, a.y);
        a.z = fmaf(w, b.z, a.z);
        a.w = fmaf(w, b.w, a.w);
    }
    __device__ static void store(float *p, const float4 &a) {
        p[0] = a.x;
        p[1] = a.y;
        p[2] = a.z;
        p[3] = a.w;
    }
};
template <>
struct Vec16<double> {
    using type = double2;
    static constexpr int n = 2;
    __device__ static double2 zero() { return make_double2(0.0, 0.0); }
    __device__ static void add(double2 &a, const double2 &b) {
        a.x += b.x;
        a.y += b.y;
    }
    __device__ static void fma(double2 &a, double w, const double2 &b) {
        a.x = ::fma(w, b.x, a.x);
        a.y = ::fma(w, b.y, a.y);
    }
    __device__ static void store(double *p, const double2 &a) {
        p[0] = a.x;
        p[1] = a.y;
    }
};

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}

// Partial Y row of (row, colouring b) over arcs [e0, e1) into ybuf[0, Wp).
template <typename T, int NV, bool WEIGHTED>
__device__ __forceinline__ void spmm_partial(const NodeArgs &A, int64_t e0, int64_t e1, int b, T *ybuf, int lane) {
    using V = Vec16<T>;
    using VT = typename V::type;
    constexpr int U = NV <= 2 ? 4 : 2;  // arcs in flight per step
    VT acc[NV];
#pragma unroll
    for (int q = 0; q < NV; ++q) acc[q] = V::zero();
    const T *Mp = static_cast<const T *>(A.Mp);
    const int64_t ldp = A.ldp;
    const int64_t nb = A.nb;
    const int nvec = (A.Wp + V::n - 1) / V::n;
    for (int64_t base = e0; base < e1; base += 32) {
        const int cnt = (int)(e1 - base < 32 ? e1 - base : 32);
        const int u_l = lane < cnt ? __ldg(A.col_idx + base + lane) : 0;
        T w_l = T(1);
        if (WEIGHTED) w_l = lane < cnt ? T(__ldg(A.weights + base + lane)) : T(0);
        int j = 0;
        for (; j + U <= cnt; j += U) {
            VT x[U][NV];
#pragma unroll
            for (int r = 0; r < U; ++r) {
                const int u = __shfl_sync(kFull, u_l, j + r);
                const VT *row = reinterpret_cast<const VT *>(Mp + ((int64_t)u * nb + b) * ldp);
#pragma unroll
                for (int q = 0; q < NV; ++q) {
                    const int vi = lane + 32 * q;
                    x[r][q] = vi < nvec ? __ldg(row + vi) : V::zero();
                }
            }
#pragma unroll
            for (int r = 0; r < U; ++r) {
                if (WEIGHTED) {
                    const T w = __shfl_sync(kFull, w_l, j + r);
#pragma unroll
                    for (int q = 0; q < NV; ++q) V::fma(acc[q], w, x[r][q]);
                } else {
#pragma unroll
                    for (int q = 0; q < NV; ++q) V::add(acc[q], x[r][q]);
                }
            }
        }
        for (; j < cnt; ++j) {
            const int u = __shfl_sync(kFull, u_l, j);
            const T w = WEIGHTED ? __shfl_sync(kFull, w_l, j) : T(1);
            const VT *row = reinterpret_cast<const VT *>(Mp + ((int64_t)u * nb + b) * ldp);
#pragma unroll
            for (int q = 0; q < NV; ++q) {
                const int vi = lane + 32 * q;
                if (vi < nvec) {
                    const VT x = __ldg(row + vi);
                    if (WEIGHTED)
                        V::fma(acc[q], w, x);
                    else
                        V::add(acc[q], x);
                }
            }
        }
    }
#pragma unroll
    for (int q = 0; q < NV; ++q) {
        const int vi = lane + 32 * q;
        if (vi < nvec) V::store(ybuf + vi * V::n, acc[q]);
    }
}

// Partial per-colour neighbour histogram of (row, colouring b) into ybuf[0, kc).
template <typename T, bool WEIGHTED>
__device__ __forceinline__ void hist_partial(const NodeArgs &A, int64_t e0, int64_t e1, int b, T *ybuf, int lane) {
    T cnt[kMaxHistColours];
#pragma unroll
    for (int c = 0; c < kMaxHistColours; ++c) cnt[c] = T(0);
    const int8_t *col = A.colours + (int64_t)b * A.n;
    for (int64_t e = e0 + lane; e < e1; e += 32) {
        const int u = __ldg(A.col_idx + e);
        const int c = __ldg(col + u);
        const T w = WEIGHTED ? T(__ldg(A.weights + e)) : T(1);
#pragma unroll
        for (int q = 0; q < kMaxHistColours; ++q) cnt[q] += (c == q) ? w : T(0);
    }
#pragma unroll
    for (int q = 0; q < kMaxHistColours; ++q) {
        if (q < A.kc) {
            const T s = warp_sum(cnt[q]);
            if (lane == 0) ybuf[q] = s;
        }
    }
}

// eMA epilogue of (row v, colouring b) from the complete Y row in ybuf.
template <typename T>
__device__ __forceinline__ void epilogue(const NodeArgs &A, int v, int b, const T *ybuf, int lane) {
    const int64_t rowb = (int64_t)v * A.nb + b;
    const int Wt = A.Wt;
    if (A.a_leaf) {
        // a colour outside [0, kc) is reported by the host after the call;
        // here it only must not index outside the gather table
        const int c = A.colours[(int64_t)b * A.n + v];
        const bool ok = (unsigned)c < (unsigned)A.kc;
        const int32_t *g = A.gather + (int64_t)(ok ? c : 0) * Wt;
        if (A.root) {
            T s = T(0);
            for (int S = lane; S < Wt; S += 32) {
                const int j = ok ? __ldg(g + S) : -1;
                if (j >= 0) s += ybuf[j];
            }
            s = warp_sum(s);
            if (lane == 0) static_cast<T *>(A.root_out)[(int64_t)b * A.n + v] = s;
        } else {
            T *out = static_cast<T *>(A.Ms) + rowb * A.ldt;
            for (int S = lane; S < Wt; S += 32) {
                const int j = ok ? __ldg(g + S) : -1;
                out[S] = j >= 0 ? ybuf[j] : T(0);
            }
        }
    } else {
        const T *ma = static_cast<const T *>(A.Ma) + rowb * A.lda;
        const int ns = A.nsplit;
        if (A.root) {
            T s = T(0);
            const int total = Wt * ns;
            for (int p = lane; p < total; p += 32) {
                const uint32_t sp = __ldg(A.splits + p);
                s = fma(__ldg(ma + (sp & 0xffffu)), ybuf[sp >> 16], s);
            }
            s = warp_sum(s);
            if (lane == 0) static_cast<T *>(A.root_out)[(int64_t)b * A.n + v] = s;
        } else {
            T *out = static_cast<T *>(A.Ms) + rowb * A.ldt;
            for (int S = lane; S < Wt; S += 32) {
                const uint32_t *sp = A.splits + (int64_t)S * ns;
                T acc = T(0);
                for (int j = 0; j < ns; ++j) {
                    const uint32_t x = __ldg(sp + j);
                    acc = fma(__ldg(ma + (x & 0xffffu)), ybuf[x >> 16], acc);
                }
                out[S] = acc;
            }
        }
    }
}

template <typename T, int NV, bool HIST, bool WEIGHTED>
__global__ void __launch_bounds__(kNodeThreads) node_kernel(const NodeArgs A) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    using V = Vec16<T>;
    constexpr int kYbuf = HIST ? kMaxHistColours : NV * 32 * V::n;
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    T *ybuf = reinterpret_cast<T *>(smem_raw) + wib * kYbuf;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t ti = (((int64_t)blockIdx.x * blockDim.x) >> 5) + wib; ti < A.ntasks; ti += nwarps) {
        const int4 task = A.tasks[ti];
        const int v = task.x;
        const int slot = task.y;
        const int64_t rs = A.row_ptr[v];
        const int64_t e0 = rs + task.z, e1 = rs + task.w;
        for (int b = 0; b < A.nb; ++b) {
            if (HIST)
                hist_partial<T, WEIGHTED>(A, e0, e1, b, ybuf, lane);
            else
                spmm_partial<T, NV, WEIGHTED>(A, e0, e1, b, ybuf, lane);
            __syncwarp();
            if (slot >= 0) {
                // one chunk of a split row: fold into the scratch row; the last
                // chunk to arrive finishes the row
                T *sc = static_cast<T *>(A.scratch) + ((int64_t)slot * A.nb + b) * A.scratch_ld;
                for (int j = lane; j < A.Wp; j += 32) atomicAdd(sc + j, ybuf[j]);
                __threadfence();
                __syncwarp();
                int last = 0;
                if (lane == 0) {
                    const unsigned done = atomicAdd(A.counters + (int64_t)slot * A.nb + b, 1u);
                    last = (done + 1u == (unsigned)__ldg(A.heavy_chunks + slot));
                }
                last = __shfl_sync(kFull, last, 0);
                if (!last) {
                    __syncwarp();
                    continue;
                }
                __threadfence();
                for (int j = lane; j < A.Wp; j += 32) ybuf[j] = __ldcg(sc + j);
                __syncwarp();
            }
            epilogue<T>(A, v, b, ybuf, lane);
            __syncwarp();
        }
    }
}

template <typename T, int NV, bool HIST, bool WEIGHTED>
void *kernel_ptr() {
    return reinterpret_cast<void *>(&node_kernel<T, NV, HIST, WEIGHTED>);
}

void *select_kernel(bool fp64, bool hist, int nv, bool weighted) {
#define SG2V_PICK(T)                                                                           \
    if (hist) return weighted ? kernel_ptr<T, 1, true, true>() : kernel_ptr<T, 1, true, false>(); \
    switch (nv) {                                                                              \
        case 1: return weighted ? kernel_ptr<T, 1, false, true>() : kernel_ptr<T, 1, false, false>(); \
        case 2: return weighted ? kernel_ptr<T, 2, false, true>() : kernel_ptr<T, 2, false, false>(); \
        case 3: return weighted ? kernel_ptr<T, 3, false, true>() : kernel_ptr<T, 3, false, false>(); \
        case 4: return weighted ? kernel_ptr<T, 4, false, true>() : kernel_ptr<T, 4, false, false>(); \
        default: return nullptr;                                                               \
    }
    if (fp64) {
        SG2V_PICK(double)
    } else {
        SG2V_PICK(float)
    }
#undef SG2V_PICK
}

// ------------------------------------------------------------- reductions

__device__ __forceinline__ void two_sum(double a, double b, double &s, double &e) {
    s = a + b;
    const double bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

__device__ __forceinline__ void rs_combine(RootSum &x, const RootSum &y) {
    const unsigned long long lo = x.lo + y.lo;
    x.hi = x.hi + y.hi + (lo < x.lo ? 1ull : 0ull);
    x.lo = lo;
    double s, e;
    two_sum(x.s, y.s, s, e);
    x.c = x.c + y.c + e;
    x.s = s;
    x.flags |= y.flags;
}

__device__ __forceinline__ RootSum rs_shfl_xor(const RootSum &x, int o) {
    RootSum y;
    y.lo = __shfl_xor_sync(kFull, x.lo, o);
    y.hi = __shfl_xor_sync(kFull, x.hi, o);
    y.s = __shfl_xor_sync(kFull, x.s, o);
    y.c = __shfl_xor_sync(kFull, x.c, o);
    y.flags = __shfl_xor_sync(kFull, x.flags, o);
    y.pad = 0;
    return y;
}

__device__ __forceinline__ RootSum rs_from(double v) {
    RootSum r;
    r.s = v;
    r.c = 0.0;
    r.lo = r.hi = 0;
    r.flags = 0;
    r.pad = 0;
    if (!isfinite(v)) {
        r.flags = kFlagNonFinite;
        r.s = 0.0;
    } else if (v != floor(v) || v < 0.0 || v >= 0x1p128) {
        r.flags = kFlagNotIntegral;
    } else if (v < 0x1p64) {
        r.lo = __double2ull_rz(v);
    } else {
        const double h = floor(v * 0x1p-64);
        r.hi = __double2ull_rz(h);
        r.lo = __double2ull_rz(v - h * 0x1p64);
    }
    return r;
}

template <typename T>
__global__ void root_partial_kernel(const T *vals, int64_t n, double *pv, RootSum *partials, int chunks) {
    __shared__ RootSum red[32];
    const int seg = blockIdx.y;
    const int chunk = blockIdx.x;
    const int64_t per = (n + chunks - 1) / chunks;
    const int64_t lo = (int64_t)chunk * per;
    const int64_t hi = (lo + per < n) ? lo + per : n;
    RootSum acc = rs_from(0.0);
    for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) {
        const double v = (double)vals[(int64_t)seg * n + i];
        if (pv) pv[(int64_t)seg * n + i] = v;
        rs_combine(acc, rs_from(v));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const RootSum y = rs_shfl_xor(acc, o);
        rs_combine(acc, y);
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) red[w] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        RootSum t = red[0];
        for (int i = 1; i < (int)(blockDim.x >> 5); ++i) rs_combine(t, red[i]);
        partials[(int64_t)seg * chunks + chunk] = t;
    }
}

__global__ void root_final_kernel(const RootSum *partials, int chunks, int nseg, RootSum *out) {
    const int seg = blockIdx.x * blockDim.x + threadIdx.x;
    if (seg >= nseg) return;
    RootSum t = partials[(int64_t)seg * chunks];
    for (int i = 1; i < chunks; ++i) rs_combine(t, partials[(int64_t)seg * chunks + i]);
    out[seg] = t;
}

__global__ void check_colours_kernel(const int8_t *colours, int64_t count, int kc, unsigned *status) {
    unsigned bad = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
        const int c = colours[i];
        bad |= (c < 0 || c >= kc) ? 1u : 0u;
    }
    bad = __any_sync(kFull, bad != 0);
    if (bad && (threadIdx.x & 31) == 0) atomicOr(status, 1u);
}

}  // namespace

size_t node_smem_bytes(bool fp64, bool hist, int nv) {
    const int vecn = fp64 ? 2 : 4;
    const size_t elems = hist ? kMaxHistColours : (size_t)nv * 32 * vecn;
    return (kNodeThreads / 32) * elems * (fp64 ? 8 : 4);
}

int node_blocks_per_sm(bool fp64, bool hist, int nv, bool weighted) {
    void *k = select_kernel(fp64, hist, nv, weighted);
    if (!k) return 0;
    int blocks = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, k, kNodeThreads, node_smem_bytes(fp64, hist, nv)) !=
        cudaSuccess)
        return 1;
    return blocks > 0 ? blocks : 1;
}

cudaError_t launch_node(const NodeArgs &args, bool fp64, int nv, int grid_cap, cudaStream_t stream) {
    const bool hist = args.hist != 0;
    const bool weighted = args.weights != nullptr;
    void *k = select_kernel(fp64, hist, nv, weighted);
    if (!k) return cudaErrorInvalidValue;
    if (args.ntasks == 0) return cudaSuccess;
    const int64_t warps_per_block = kNodeThreads / 32;
    int64_t grid = (args.ntasks + warps_per_block - 1) / warps_per_block;
    if (grid > grid_cap) grid = grid_cap;
    if (grid < 1) grid = 1;
    NodeArgs a = args;
    void *params[] = {&a};
    return cudaLaunchKernel(k, dim3((unsigned)grid), dim3(kNodeThreads), params, node_smem_bytes(fp64, hist, nv),
                            stream);
}

cudaError_t launch_root_reduce(const void *vals, bool fp64, int64_t n, int nseg, double *pv, RootSum *partials,
                               int chunks, RootSum *out, cudaStream_t stream) {
    dim3 grid((unsigned)chunks, (unsigned)nseg);
    if (fp64)
        root_partial_kernel<double><<<grid, 256, 0, stream>>>(static_cast<const double *>(vals), n, pv, partials,
                                                                chunks);
    else
        root_partial_kernel<float><<<grid, 256, 0, stream>>>(static_cast<const float *>(vals), n, pv, partials,
                                                               chunks);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    root_final_kernel<<<(nseg + 127) / 128, 128, 0, stream>>>(partials, chunks, nseg, out);
    return cudaGetLastError();
}

cudaError_t launch_check_colours(const int8_t *colours, int64_t count, int kc, unsigned *status,
                                 cudaStream_t stream) {
    if (count == 0) return cudaSuccess;
    int64_t blocks = (count + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    check_colours_kernel<<<(unsigned)blocks, 256, 0, stream>>>(colours, count, kc, status);
    return cudaGetLastError();
}

}  // namespace sg2v
