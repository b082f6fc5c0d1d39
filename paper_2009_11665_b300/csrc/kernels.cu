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

#include <algorithm>
#include <cstdint>
#include <map>
#include <mutex>
#include <tuple>
#include <type_traits>
#include <unordered_map>

#include "device_common.cuh"
#include "kernels.cuh"

namespace sg2v {

namespace {

// FORM selects a specialised epilogue (chosen on the host by node_form):
// 0 generic; 1 single-vertex active child with a plain output row (the
// expansion writes M_s' = Y' straight to the table); 2 a root with one
// output set (rootpair: each lane pairs its p-sets with their active sets,
// no Y' in shared memory).
template <typename T, int G, int NV, bool HIST, bool WEIGHTED, bool SCALED, int FORM>
__global__ void __launch_bounds__(kNodeThreads, MinBlocks<T, NV>::value) node_kernel(const NodeArgs A) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    T *zbuf = reinterpret_cast<T *>(smem_raw) + (int64_t)wib * (A.zwords + A.ywords + A.mwords + A.owords);
    T *ybuf = zbuf + A.zwords;
    T *mbuf = ybuf + A.ywords;  // this row's active-child row (a >= 2)
    T *obuf = mbuf + A.mwords;  // this row's outputs before normalisation (scaled)
    const int zlen = HIST ? A.kc : A.kc * A.wz_pad;
    const int mchunks = (A.a_leaf || A.defer) ? 0 : (A.Wa * (int)sizeof(T) + 15) / 16;
    constexpr bool direct = FORM == 1 && !SCALED;
    constexpr bool pairs = FORM == 2 && !SCALED && !HIST;
    uint16_t pr[4] = {0, 0, 0, 0};
    if constexpr (pairs) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int j = lane + 32 * q;
            pr[q] = j < A.wy ? __ldg(A.rootpair + j) : (uint16_t)0;
        }
    }
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    int64_t ti = (((int64_t)blockIdx.x * blockDim.x) >> 5) + wib;
    int4 task = ti < A.ntasks ? A.tasks[ti] : make_int4(0, -1, 0, 0);
    unsigned ovf = 0;
    for (; ti < A.ntasks; ti += nwarps) {
        // the next task's descriptor is fetched while this one runs
        const int4 next = ti + nwarps < A.ntasks ? A.tasks[ti + nwarps] : task;
        const int v = task.x;
        const int slot = task.y;
        const int64_t e0 = task.z, e1 = task.w;
        for (int b = 0; b < A.nb; ++b) {
            const int cv = A.colours[(int64_t)b * A.n + v];
            const bool cok = (unsigned)cv < (unsigned)A.kc;
            if (e0 == e1 && A.defer) {
                T *yo = static_cast<T *>(A.Yout) + ((int64_t)v * A.nb + b) * A.ldy;
                for (int j = lane; j < A.wy; j += 32) yo[j] = T(0);
                continue;
            }
            if (e0 == e1) {
                // no arcs: Y' = 0, so every output of the row is zero
                if constexpr (SCALED)
                    epilogue_scaled(A, v, b, false, ybuf, mbuf, obuf, 0, lane);
                else
                    epilogue<T>(A, v, b, false, ybuf, mbuf, lane, ovf);
                continue;
            }
            int eref = 0;
            if (SCALED && !HIST) eref = row_eref(A, (int64_t)v * A.nb + b);
            if (mchunks && cok) {
                // start copying the active row now; it is needed only by the eMA
                const char *src = static_cast<const char *>(A.Ma) + ((int64_t)v * A.nb + b) * A.lda * sizeof(T);
                for (int c = lane; c < mchunks; c += 32) {
                    const unsigned dst = (unsigned)__cvta_generic_to_shared(reinterpret_cast<char *>(mbuf) + 16 * c);
                    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(dst), "l"(src + 16 * c) : "memory");
                }
                asm volatile("cp.async.commit_group;\n" ::: "memory");
            }
            if (HIST)
                hist_z<T, WEIGHTED>(A, e0, e1, b, zbuf, lane);
            else
                spmm_z<T, G, NV, WEIGHTED, SCALED>(A, v, e0, e1, b, cv, eref, zbuf, lane, ovf);
            __syncwarp();
            if (slot >= 0) {
                // one chunk of a split row: fold Z into the scratch row; the
                // last chunk to arrive finishes the row
                T *sc = static_cast<T *>(A.scratch) + ((int64_t)slot * A.nb + b) * A.scratch_ld;
                // (the row of v's own colour in Z is stale and read by nothing)
                const int own0 = HIST ? zlen : cv * A.wz_pad, own1 = HIST ? zlen : own0 + A.wz_pad;
                for (int j = lane; j < zlen; j += 32)
                    if (j < own0 || j >= own1) atomic_add(sc + j, zbuf[j], ovf);
                __threadfence();
                __syncwarp();
                int last = 0;
                if (lane == 0) {
                    const unsigned done = atomicAdd(A.counters + (int64_t)slot * A.nb + b, 1u);
                    last = (done + 1u == (unsigned)__ldg(A.heavy_chunks + slot));
                }
                last = __shfl_sync(kFull, last, 0);
                if (!last) {
                    if (mchunks && cok) asm volatile("cp.async.wait_all;\n" ::: "memory");
                    __syncwarp();
                    continue;
                }
                __threadfence();
                for (int j = lane; j < zlen; j += 32) zbuf[j] = __ldcg(sc + j);
                __syncwarp();
            }
            if constexpr (pairs) {
                // row sum = sum over p-sets P' of M_a'(S' - P') * Y'(P')
                if (mchunks && cok) asm volatile("cp.async.wait_all;\n" ::: "memory");
                __syncwarp();
                T s = T(0);
                if (cok) {
                    const uint16_t *ex = A.expand + (int64_t)cv * A.wy * A.pstride;
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const int j = lane + 32 * q;
                        if (j < A.wy) Ar<T>::mad(s, mbuf[pr[q]], expand_set(ex, A.pstride, A.p, j, zbuf, ovf), ovf);
                    }
                }
                s = group_sum_chk<32>(s, ovf);
                if (lane == 0)
                    static_cast<T *>(A.root_out)[(int64_t)b * A.n + v] = A.half_arcs ? Ar<T>::twice(s, ovf) : s;
                __syncwarp();
                continue;
            }
            if constexpr (direct) {
                // M_s' = Y': straight from the expansion to the output row
                T *out = static_cast<T *>(A.Ms) + ((int64_t)v * A.nb + b) * A.ldt;
                if (cok)
                    expand_y<T>(A, cv, zbuf, out, lane, ovf);
                else
                    for (int j = lane; j < A.Ws; j += 32) out[j] = T(0);
                __syncwarp();
                continue;
            }
            if (cok) expand_y<T>(A, cv, zbuf, ybuf, lane, ovf);
            if (mchunks && cok) asm volatile("cp.async.wait_all;\n" ::: "memory");
            __syncwarp();
            if (A.defer) {
                // the eMA runs in its own launch over blocks of rows
                T *yo = static_cast<T *>(A.Yout) + ((int64_t)v * A.nb + b) * A.ldy;
                for (int j = lane; j < A.wy; j += 32) yo[j] = cok ? ybuf[j] : T(0);
                __syncwarp();
                continue;
            }
            if constexpr (SCALED) {
                const int base = (A.a_leaf ? 0 : (int)A.Ea[(int64_t)v * A.nb + b]) + eref;
                epilogue_scaled(A, v, b, cok, ybuf, mbuf, obuf, base, lane);
            } else {
                epilogue<T>(A, v, b, cok, ybuf, mbuf, lane, ovf);
            }
            __syncwarp();
        }
        report_ovf<T>(A.status, ovf);
        task = next;
    }
}

// Narrow rows (G = 4, 8 or 16 lanes cover a compressed row): every group of
// G lanes of a warp takes its own work-list task, so a warp runs 32 / G rows
// at once and the per-row chain (colour, arc batch, gathers, expansion,
// epilogue) is paid once per 32 / G rows.  A group walks its row's sorted
// arcs in batches of G, compacted to the arcs that add something; groups
// step together (the warp runs to its longest row, shorter rows read the
// zero row).  Shared memory per group: Z [kc][wz_pad], Y', the active row
// and (scaled) the output row.  FORM 1 (single-vertex active child, plain
// output): the expansion writes M_s' = Y' straight to the output row.
template <typename T, int G, bool WEIGHTED, bool SCALED, int FORM = 0>
__global__ void __launch_bounds__(kNodeThreads, MinBlocks<T, 1>::value) node_group_kernel(const NodeArgs A) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    using V = Vec16<T>;
    using VT = typename V::type;
    constexpr int NG = 32 / G;
    constexpr int U = 4;                       // arcs in flight per group and step
    constexpr bool FMA = WEIGHTED || SCALED;
    constexpr bool SKIP_ZERO = sizeof(T) >= 8;
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int grp = lane / G, gl = lane % G, g0 = grp * G;
    const unsigned gbits = (G == 32 ? kFull : ((1u << G) - 1u)) << g0;
    const int kc = A.kc, wzp = A.wz_pad;       // wzp = G * V::n
    const int per_group = kc * wzp + A.ywords + A.mwords + A.owords;
    T *zg = reinterpret_cast<T *>(smem_raw) + (int64_t)(wib * NG + grp) * per_group;
    T *ybuf = zg + kc * wzp;
    T *mbuf = ybuf + A.ywords;
    T *obuf = mbuf + A.mwords;
    const int mchunks = (A.a_leaf || A.defer) ? 0 : (A.Wa * (int)sizeof(T) + 15) / 16;
    const bool qok = gl < (A.Wz + V::n - 1) / V::n;
    const bool zok = gl < wzp / V::n;  // Z rows hold wzp / V::n vectors
    // integer tables of odd width: the last vector's padding element is cleared
    const bool tail = Ar<T>::exact && V::n == 2 && (A.Wz & 1) && gl == (A.Wz + V::n - 1) / V::n - 1;
    const int zero_row = (int)A.n;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t wglob = (((int64_t)blockIdx.x * blockDim.x) >> 5) + wib;
    const int64_t nrounds = (A.ntasks + (int64_t)NG - 1) / NG;
    unsigned ovf = 0;
    for (int64_t rnd = wglob; rnd < nrounds; rnd += nwarps) {
        const int64_t ti = rnd * NG + grp;
        const bool have = ti < A.ntasks;
        const int4 task = have ? A.tasks[ti] : make_int4(0, -1, 0, 0);
        const int v = task.x, slot = task.y;
        const int e0 = task.z, e1 = task.w;
        // batches of G arcs of the longest row in the warp
        const int nbat_w = __reduce_max_sync(kFull, (unsigned)((e1 - e0 + G - 1) / G));
        for (int b = 0; b < A.nb; ++b) {
            const int64_t rowb = (int64_t)v * A.nb + b;
            const int cv = have ? (int)A.colours[(int64_t)b * A.n + v] : -1;
            const bool cok = have && (unsigned)cv < (unsigned)kc;
            const int eref = (SCALED && have) ? row_eref(A, rowb) : 0;
            if (mchunks && cok) {
                const char *src = static_cast<const char *>(A.Ma) + rowb * A.lda * sizeof(T);
                for (int c = gl; c < mchunks; c += G) {
                    const unsigned dst = (unsigned)__cvta_generic_to_shared(reinterpret_cast<char *>(mbuf) + 16 * c);
                    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(dst), "l"(src + 16 * c) : "memory");
                }
            }
            asm volatile("cp.async.commit_group;\n" ::: "memory");
            const VT *Mb = reinterpret_cast<const VT *>(static_cast<const T *>(A.Mp) + (int64_t)b * A.ldp) + gl;
            const int64_t uvec = (int64_t)A.nb * A.ldp / V::n;
            const int32_t *scol = A.scol + (int64_t)b * A.nnz;
            const int8_t *sclr = A.sclr + (int64_t)b * A.nnz;
            const float *sw = WEIGHTED ? A.sw + (int64_t)b * A.nnz : nullptr;
            const int16_t *Ep = SCALED ? A.Ep + b : nullptr;
            VT run = V::zero();
            int cur = -1;
            uint32_t seen = 0;
            auto flush = [&](int c) {
                if (c != cv) {
                    if (zok) reinterpret_cast<VT *>(zg + c * wzp)[gl] = run;
                    seen |= 1u << c;
                }
                run = V::zero();
            };
            for (int kb = 0; kb < nbat_w; ++kb) {
                const int base = e0 + kb * G;
                const bool in = base + gl < e1;
                const int c_in = in ? (int)__ldg(sclr + base + gl) : -1;
                bool t_in = c_in >= 0 && c_in != cv;
                const int u_in = t_in ? __ldg(scol + base + gl) : zero_row;
                if (A.half_arcs && u_in >= v) t_in = false;
                const unsigned live = (__ballot_sync(kFull, t_in) & gbits) >> g0;
                const int cnt = __popc(live);
                const int cnt_w = __reduce_max_sync(kFull, (unsigned)cnt);
                const bool t_l = gl < cnt;
                const int src = g0 + (t_l ? (int)__fns(live, 0, gl + 1) : gl);
                int u_l = __shfl_sync(kFull, u_in, src);
                int c_l = __shfl_sync(kFull, c_in, src);
                const int c_last = __shfl_sync(kFull, c_l, g0 + (cnt > 0 ? cnt - 1 : 0));
                if (!t_l) {
                    u_l = zero_row;
                    c_l = cnt > 0 ? c_last : (cur >= 0 ? cur : 0);
                }
                T w_l = T(1);
                if (WEIGHTED) w_l = t_l ? T(__ldg(sw + base + (src - g0))) : T(0);
                int ep_l = eref;
                if (SCALED && t_l) ep_l = (int)__ldg(Ep + (int64_t)u_l * A.nb);
                for (int j0 = 0; j0 < cnt_w; j0 += U) {
                    VT x[U];
                    T w[U];
                    int cr[U];
                    bool lv[U];
#pragma unroll
                    for (int r = 0; r < U; ++r) {
                        const int j = (j0 + r) & (G - 1);
                        const bool inb = j0 + r < G;
                        const int u = __shfl_sync(kFull, u_l, g0 + j);
                        cr[r] = __shfl_sync(kFull, c_l, g0 + j);
                        lv[r] = inb && j0 + r < cnt && (!SKIP_ZERO || u != zero_row);
                        w[r] = WEIGHTED ? __shfl_sync(kFull, w_l, g0 + j) : T(1);
                        if (SCALED) {
                            const int ep = __shfl_sync(kFull, ep_l, g0 + j);
                            w[r] *= T(exp2_neg(ep - eref));
                        }
                        const VT *row = Mb + (int64_t)(lv[r] ? u : zero_row) * uvec;
                        x[r] = (SKIP_ZERO ? (lv[r] && qok) : (qok || !A.pred_lanes)) ? ldg_row(row) : V::zero();
                        if constexpr (Ar<T>::exact && V::n == 2)
                            if (tail) x[r].y = 0;
                    }
#pragma unroll
                    for (int r = 0; r < U; ++r) {
                        if (!lv[r]) continue;
                        if (cr[r] != cur) {
                            if (cur >= 0) flush(cur);
                            cur = cr[r];
                        }
                        if (FMA)
                            V::fma(run, w[r], x[r]);
                        else
                            vadd<T>(run, x[r], ovf);
                    }
                }
            }
            if (cur >= 0) flush(cur);
            for (int d = 0; d < kc; ++d)
                if (!(seen >> d & 1u) && d != cv && zok) reinterpret_cast<VT *>(zg + d * wzp)[gl] = V::zero();
            __syncwarp();
            // split rows: fold Z into the scratch row; the last chunk finishes
            bool fin = have;
            if (have && slot >= 0) {
                T *sc = static_cast<T *>(A.scratch) + ((int64_t)slot * A.nb + b) * A.scratch_ld;
                // (the row of v's own colour in Z is stale and read by nothing)
                for (int j = gl; j < kc * wzp; j += G)
                    if (j / wzp != cv) atomic_add(sc + j, zg[j], ovf);
                __threadfence();
            }
            __syncwarp();
            int last = 1;
            if (have && slot >= 0 && gl == 0) {
                const unsigned done = atomicAdd(A.counters + (int64_t)slot * A.nb + b, 1u);
                last = done + 1u == (unsigned)__ldg(A.heavy_chunks + slot);
            }
            last = __shfl_sync(kFull, last, g0);
            if (have && slot >= 0) {
                fin = last != 0;
                if (fin) {
                    __threadfence();
                    T *sc = static_cast<T *>(A.scratch) + ((int64_t)slot * A.nb + b) * A.scratch_ld;
                    for (int j = gl; j < kc * wzp; j += G) zg[j] = __ldcg(sc + j);
                }
            }
            __syncwarp();
            const bool ok = fin && cok && e0 < e1;
            if constexpr (FORM == 1 && !SCALED) {
                if (fin) {
                    T *out = static_cast<T *>(A.Ms) + rowb * A.ldt;
                    const uint16_t *ex = A.expand + (int64_t)(ok ? cv : 0) * A.wy * A.pstride;
                    for (int j = gl; j < A.wy; j += G)
                        out[j] = ok ? expand_set(ex, A.pstride, A.p, j, zg, ovf) : T(0);
                }
                __syncwarp();
                continue;
            }
            if (ok) {
                const uint16_t *ex = A.expand + (int64_t)cv * A.wy * A.pstride;
                for (int j = gl; j < A.wy; j += G) ybuf[j] = expand_set(ex, A.pstride, A.p, j, zg, ovf);
            }
            asm volatile("cp.async.wait_all;\n" ::: "memory");
            __syncwarp();
            if (fin && (A.defer || (!SCALED && A.Yout))) {
                T *yo = static_cast<T *>(A.Yout) + rowb * A.ldy;
                for (int j = gl; j < A.wy; j += G) yo[j] = ok ? ybuf[j] : T(0);
            }
            if (A.defer) {
                __syncwarp();
                continue;
            }
            // eMA epilogue of the group's row
            const int base_e = SCALED ? (A.a_leaf ? 0 : (fin && have ? (int)A.Ea[rowb] : 0)) + eref : 0;
            if (A.root) {
                const T sum = group_sum_chk<G>(ema_root_partial<T, G>(A, ok, ybuf, mbuf, gl, ovf), ovf);
                if (fin && gl == 0) {
                    if constexpr (SCALED)
                        A.root_out_d[(int64_t)b * A.n + v] = ok ? ldexp((double)sum, base_e + (A.half_arcs ? 1 : 0)) : 0.0;
                    else
                        static_cast<T *>(A.root_out)[(int64_t)b * A.n + v] = A.half_arcs ? Ar<T>::twice(sum, ovf) : sum;
                }
            } else if constexpr (SCALED) {
                T mx = T(0);
                ema_rows<T, G>(A, ok, ybuf, mbuf, gl, ovf, [&](int S, T x) {
                    obuf[S] = x;
                    mx = fmax(mx, x);
                });
                mx = group_max<G>(mx);
                const int em = mx > T(0) ? ilogb(mx) : 0;
                __syncwarp();
                if (fin) {
                    T *out = static_cast<T *>(A.Ms) + rowb * A.ldt;
                    for (int j = gl; j < A.Ws; j += G) out[j] = ldexp(obuf[j], -em);
                    if (gl == 0) A.Es[rowb] = mx > T(0) ? clamp_exp(base_e + em) : kEmptyRowExp;
                }
            } else {
                T *out = static_cast<T *>(A.Ms) + rowb * A.ldt;
                const bool accumulate = A.accumulate != 0;
                ema_rows<T, G>(A, ok, ybuf, mbuf, gl, ovf, [&](int S, T x) {
                    if (!fin) return;
                    if (accumulate) Ar<T>::add(x, out[S], ovf);
                    out[S] = x;
                });
            }
            __syncwarp();
        }
        report_ovf<T>(A.status, ovf);
    }
}

// Histogram nodes (passive child a single vertex) in blocks of 32 rows per
// warp: first every lane counts the neighbour colours of its own row (the
// arcs of neighbouring work-list tasks have similar lengths), then the warp
// runs the expansion and eMA epilogue of the 32 rows one after another.  The
// per-row chain of dependent loads of the one-warp-per-row kernel is paid
// once per 32 rows.  Shared memory per warp: counts [kc][32], the active rows
// of the block [32][mwords], Y' and (scaled) the output row.
constexpr int kHistRows = 32;
// rows with at most this many eMA products run their epilogue one per lane
constexpr int kLaneRowProducts = 1024;

template <typename T, bool WEIGHTED, bool SCALED>
__global__ void __launch_bounds__(kNodeThreads, 4) hist_rows_kernel(const NodeArgs A) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const int kc = A.kc;
    const int per_warp = kc * kHistRows + kHistRows * A.mwords + A.ywords + A.owords;
    T *cnt = reinterpret_cast<T *>(smem_raw) + (int64_t)wib * per_warp;  // [kc][32]
    T *mrows = cnt + kc * kHistRows;                                      // [32][mwords]
    T *ybuf = mrows + kHistRows * A.mwords;
    T *obuf = ybuf + A.ywords;
    const int mchunks = A.a_leaf ? 0 : (A.Wa * (int)sizeof(T) + 15) / 16;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t nblocks = (A.ntasks + kHistRows - 1) / kHistRows;
    unsigned ovf = 0;
    for (int64_t blk = (((int64_t)blockIdx.x * blockDim.x) >> 5) + wib; blk < nblocks; blk += nwarps) {
        const int64_t t = blk * kHistRows + lane;
        const bool have = t < A.ntasks;
        const int4 task = have ? A.tasks[t] : make_int4(0, -1, 0, 0);
        for (int b = 0; b < A.nb; ++b) {
            // the active rows of the block's rows, copied while the counts run
            if (mchunks) {
                for (int r = 0; r < kHistRows; ++r) {
                    const int vr = __shfl_sync(kFull, task.x, r);
                    const bool hr = __shfl_sync(kFull, (int)have, r) != 0;
                    if (!hr) continue;
                    const char *src =
                        static_cast<const char *>(A.Ma) + ((int64_t)vr * A.nb + b) * A.lda * sizeof(T);
                    char *dst = reinterpret_cast<char *>(mrows + r * A.mwords);
                    for (int c = lane; c < mchunks; c += 32) {
                        const unsigned d = (unsigned)__cvta_generic_to_shared(dst + 16 * c);
                        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src + 16 * c)
                                     : "memory");
                    }
                }
                asm volatile("cp.async.commit_group;\n" ::: "memory");
            }
            // phase 1: lane = row, counts of neighbour colours (and the row's
            // own colour and active-row exponent, for phase 2)
            const int cv_l = have ? (int)A.colours[(int64_t)b * A.n + task.x] : -1;
            const int ea_l = (SCALED && have && !A.a_leaf) ? (int)A.Ea[(int64_t)task.x * A.nb + b] : 0;
            const int8_t *sclr = A.sclr + (int64_t)b * A.nnz;
            const float *sw = WEIGHTED ? A.sw + (int64_t)b * A.nnz : nullptr;
            // counts written by the colour sort (the whole row's, also for
            // split rows, whose first chunk then finishes the row alone)
            const bool sorted_counts = !WEIGHTED && A.hcount != nullptr;
            if (sorted_counts) {
                const int32_t *hr = A.hcount + ((int64_t)task.x * A.nb + b) * A.hld;
                for (int d = 0; d < kc; ++d) cnt[d * kHistRows + lane] = have ? T(__ldg(hr + d)) : T(0);
            } else {
                for (int d = 0; d < kc; ++d) cnt[d * kHistRows + lane] = T(0);
            }
            if (sorted_counts) {
                // loaded above
            } else if (WEIGHTED) {
                // eight arcs per step: their loads issue together
                for (int64_t e = task.z; e < task.w; e += 8) {
                    int c[8];
                    T w[8];
#pragma unroll
                    for (int k = 0; k < 8; ++k) {
                        const bool in = e + k < task.w;
                        c[k] = in ? (int)__ldg(sclr + e + k) : -1;
                        w[k] = in ? T(__ldg(sw + e + k)) : T(0);
                    }
#pragma unroll
                    for (int k = 0; k < 8; ++k)
                        if (c[k] >= 0) cnt[c[k] * kHistRows + lane] += w[k];
                }
            } else {
                // the row's colours in aligned 16-byte words (the colour
                // buffer is padded by 16 bytes at both ends)
                const uintptr_t lo = reinterpret_cast<uintptr_t>(sclr + task.z);
                const uintptr_t hi = reinterpret_cast<uintptr_t>(sclr + task.w);
                for (uintptr_t a = lo & ~uintptr_t(15); a < hi; a += 16) {
                    const uint4 q = __ldg(reinterpret_cast<const uint4 *>(a));
                    const uint32_t wds[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
                    for (int k = 0; k < 16; ++k) {
                        const uintptr_t at = a + k;
                        const int c = (int)(int8_t)(wds[k >> 2] >> (8 * (k & 3)));
                        if (at >= lo && at < hi && c >= 0) cnt[c * kHistRows + lane] += T(1);
                    }
                }
            }
            // split rows: fold the chunk's counts; the last chunk finishes the row
            bool finish = have;
            if (sorted_counts) {
                if (have && task.y >= 0) finish = (int64_t)task.z == __ldg(A.row_ptr + task.x);
            } else if (have && task.y >= 0) {
                T *sc = static_cast<T *>(A.scratch) + ((int64_t)task.y * A.nb + b) * A.scratch_ld;
                for (int d = 0; d < kc; ++d) atomic_add(sc + d, cnt[d * kHistRows + lane], ovf);
                __threadfence();
                const unsigned done = atomicAdd(A.counters + (int64_t)task.y * A.nb + b, 1u);
                finish = done + 1u == (unsigned)__ldg(A.heavy_chunks + task.y);
                if (finish) {
                    __threadfence();
                    for (int d = 0; d < kc; ++d) cnt[d * kHistRows + lane] = __ldcg(sc + d);
                }
            }
            const unsigned fin = __ballot_sync(kFull, finish);
            if (mchunks) asm volatile("cp.async.wait_all;\n" ::: "memory");
            __syncwarp();
            if ((int64_t)A.Ws * (A.a_leaf ? 1 : A.nsplit) <= kLaneRowProducts) {
                // phase 2 for small rows: lane = row as well.  With a single-
                // vertex passive child, Y'(j) is the count of the j-th colour
                // other than v's own.
                const bool mine = (fin >> lane & 1u) != 0;
                const int cv = cv_l;
                const bool ok = mine && (unsigned)cv < (unsigned)kc && task.w > task.z;
                const int64_t rowb = (int64_t)task.x * A.nb + b;
                auto y = [&](int j) -> T { return cnt[(j < cv ? j : j + 1) * kHistRows + lane]; };
                const T *ma = mrows + lane * A.mwords;
                if (mine && A.Yout && !SCALED) {
                    T *yo = static_cast<T *>(A.Yout) + rowb * A.ldy;
                    for (int j = 0; j < A.wy; ++j) yo[j] = ok ? y(j) : T(0);
                }
                T sum = T(0), mx = T(0);
                T *out = A.root ? nullptr : static_cast<T *>(A.Ms) + rowb * A.ldt;
                for (int S = 0; S < A.Ws; ++S) {
                    T acc = T(0);
                    if (ok) {
                        if (A.a_leaf) {
                            acc = y(S);
                        } else {
                            const uint32_t *sp = A.splits + (int64_t)S * A.nsplit;
                            for (int j = 0; j < A.nsplit; ++j) {
                                const uint32_t x = __ldg(sp + j);
                                Ar<T>::mad(acc, ma[x & 0xffffu], y((int)(x >> 16)), ovf);
                            }
                        }
                    }
                    Ar<T>::add(sum, acc, ovf);
                    if constexpr (SCALED) mx = fmax(mx, acc);
                    if (out && mine) {
                        if (!SCALED && A.accumulate) Ar<T>::add(acc, out[S], ovf);
                        out[S] = acc;
                    }
                }
                if (mine) {
                    if constexpr (SCALED) {
                        const int base = ea_l;
                        if (A.root) {
                            A.root_out_d[(int64_t)b * A.n + task.x] = ok ? ldexp((double)sum, base) : 0.0;
                        } else {
                            const int em = mx > T(0) ? ilogb(mx) : 0;
                            if (em != 0)
                                for (int S = 0; S < A.Ws; ++S) out[S] = ldexp(out[S], -em);
                            A.Es[rowb] = mx > T(0) ? clamp_exp(base + em) : kEmptyRowExp;
                        }
                    } else if (A.root) {
                        static_cast<T *>(A.root_out)[(int64_t)b * A.n + task.x] = sum;
                    }
                }
                __syncwarp();
                continue;
            }
            // phase 2: warp = row, expansion and eMA epilogue
            for (int r = 0; r < kHistRows; ++r) {
                if (!(fin >> r & 1u)) continue;
                const int v = __shfl_sync(kFull, task.x, r);
                const int cv = __shfl_sync(kFull, cv_l, r);
                const bool cok = (unsigned)cv < (unsigned)kc;
                const bool arcs = __shfl_sync(kFull, task.w - task.z, r) > 0;
                if (cok) {
                    const uint16_t *ex = A.expand + (int64_t)cv * A.wy;
                    for (int j = lane; j < A.wy; j += 32) ybuf[j] = cnt[(int)__ldg(ex + j) * kHistRows + r];
                }
                __syncwarp();
                const T *ma = mrows + r * A.mwords;
                const bool ok = cok && arcs;
                if constexpr (SCALED) {
                    const int base = __shfl_sync(kFull, ea_l, r);
                    epilogue_scaled(A, v, b, ok, ybuf, ma, obuf, base, lane);
                } else {
                    epilogue<T>(A, v, b, ok, ybuf, ma, lane, ovf);
                }
                __syncwarp();
            }
        }
        report_ovf<T>(A.status, ovf);
    }
}

// Deferred eMA over blocks of kEmaRows rows (rows r0 .. r0 + R - 1 of the
// flattened (vertex, colouring) row space).  Shared memory holds the block's
// Y' and active rows interleaved by row ([index][R]), so one split word and
// short vector loads give R products.  Scaled outputs are stored as they
// are, then rescaled in place once the block knows each row's largest value.
template <typename T>
struct RowVec;
template <>
struct RowVec<float> {
    static __device__ void load(const float *p, float (&x)[kEmaRows]) {
#pragma unroll
        for (int i = 0; i < kEmaRows; i += 4) {
            const float4 v = *reinterpret_cast<const float4 *>(p + i);
            x[i] = v.x; x[i + 1] = v.y; x[i + 2] = v.z; x[i + 3] = v.w;
        }
    }
};
template <>
struct RowVec<double> {
    static __device__ void load(const double *p, double (&x)[kEmaRows]) {
#pragma unroll
        for (int i = 0; i < kEmaRows; i += 2) {
            const double2 a = *reinterpret_cast<const double2 *>(p + i);
            x[i] = a.x; x[i + 1] = a.y;
        }
    }
};
template <>
struct RowVec<u128> {
    static __device__ void load(const u128 *p, u128 (&x)[kEmaRows]) {
#pragma unroll
        for (int i = 0; i < kEmaRows; ++i) x[i] = p[i];
    }
};
template <>
struct RowVec<u64> {
    static __device__ void load(const u64 *p, u64 (&x)[kEmaRows]) {
#pragma unroll
        for (int i = 0; i < kEmaRows; i += 2) {
            const ulonglong2 a = *reinterpret_cast<const ulonglong2 *>(p + i);
            x[i] = a.x; x[i + 1] = a.y;
        }
    }
};
static_assert(kEmaRows % 4 == 0, "RowVec loads rows four at a time");

template <typename T, bool SCALED>
__global__ void __launch_bounds__(256) ema_rows_kernel(const NodeArgs A) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr int R = kEmaRows;
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const int wy = A.wy, wa = A.Wa, ws = A.Ws, ns = A.nsplit;
    T *ys = reinterpret_cast<T *>(smem_raw);            // [wy][R]
    T *mas = ys + (int64_t)wy * R;                       // [wa][R]
    __shared__ T s_max[R][8];
    __shared__ int s_ok[R];
    const int64_t rows = A.live_rows * A.nb;
    unsigned ovf = 0;
    for (int64_t r0 = (int64_t)blockIdx.x * R; r0 < rows; r0 += (int64_t)gridDim.x * R) {
        if (tid < R) {
            const int64_t row = r0 + tid;
            bool ok = row < rows;
            if (ok) {
                const int64_t v = row / A.nb, b = row - v * A.nb;
                ok = (unsigned)A.colours[b * A.n + v] < (unsigned)A.kc;
            }
            s_ok[tid] = ok;
        }
        for (int i = tid; i < R * wy; i += blockDim.x) {
            const int r = i / wy, j = i - r * wy;
            const int64_t row = r0 + r;
            ys[j * R + r] = row < rows ? static_cast<const T *>(A.Yout)[row * A.ldy + j] : T(0);
        }
        for (int i = tid; i < R * wa; i += blockDim.x) {
            const int r = i / wa, j = i - r * wa;
            const int64_t row = r0 + r;
            mas[j * R + r] = row < rows ? static_cast<const T *>(A.Ma)[row * A.lda + j] : T(0);
        }
        __syncthreads();
        T mx[R];
#pragma unroll
        for (int r = 0; r < R; ++r) mx[r] = T(0);
        for (int S = tid; S < ws; S += blockDim.x) {
            T acc[R];
#pragma unroll
            for (int r = 0; r < R; ++r) acc[r] = T(0);
            const uint32_t *sp = A.splits + (int64_t)S * ns;
            for (int j = 0; j < ns; ++j) {
                const uint32_t x = __ldg(sp + j);
                T m[R], y[R];
                RowVec<T>::load(mas + (x & 0xffffu) * R, m);
                RowVec<T>::load(ys + (x >> 16) * R, y);
#pragma unroll
                for (int r = 0; r < R; ++r) Ar<T>::mad(acc[r], m[r], y[r], ovf);
            }
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const T val = s_ok[r] ? acc[r] : T(0);
                if constexpr (SCALED) mx[r] = fmax(mx[r], val);
                if (r0 + r < rows) static_cast<T *>(A.Ms)[(r0 + r) * A.ldt + S] = val;
            }
        }
        if constexpr (SCALED) {
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const T m = warp_max(mx[r]);
                if (lane == 0) s_max[r][w] = m;
            }
            __syncthreads();
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const int64_t row = r0 + r;
                if (row >= rows) continue;
                T m = T(0);
                for (int i = 0; i < (int)(blockDim.x >> 5); ++i) m = fmax(m, s_max[r][i]);
                const int em = m > T(0) ? ilogb(m) : 0;
                T *out = static_cast<T *>(A.Ms) + row * A.ldt;
                // the same thread wrote out[S] above
                if (em != 0)
                    for (int S = tid; S < ws; S += blockDim.x) out[S] = ldexp(out[S], -em);
                if (tid == 0) {
                    const int base = (int)A.Ea[row] + row_eref(A, row);
                    A.Es[row] = m > T(0) ? clamp_exp(base + em) : kEmptyRowExp;
                }
            }
        }
        __syncthreads();
        report_ovf<T>(A.status, ovf);
    }
}

// Wide rows (a compressed row wider than one warp's register tile): one
// 256-thread CTA per (task, colouring).  Warp w owns vectors
// [w*32*NV, (w+1)*32*NV) of every gathered row and of Z(d, .), so the eight
// warps walk the same colour-sorted arc list over disjoint column slices; the
// expansion, the eMA and the root's row sum then use all threads.
constexpr int kWideWarps = 8;
static_assert(kWideWarps * 32 == kWideThreads, "wide CTA size");

template <typename T, int NV, bool WEIGHTED, bool SCALED>
__global__ void __launch_bounds__(kWideWarps * 32, 1) node_wide_kernel(const NodeArgs A) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    using V = Vec16<T>;
    using VT = typename V::type;
    constexpr int U = NV == 1 ? 4 : 2;
    static_assert(32 % U == 0, "a step's arcs must stay inside one batch of 32");
    constexpr bool FMA = WEIGHTED || SCALED;
    __shared__ int s_last;
    __shared__ T s_red[kWideWarps];
    __shared__ T s_max[kWideWarps];
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const int kc = A.kc, wzp = A.wz_pad;  // wzp = the row's vectors * V::n
    // Z in shared memory, or (rows too wide for it) in this CTA's slot of a
    // global scratch that stays in L2
    T *zbuf = A.zglobal ? static_cast<T *>(A.zglobal) + (int64_t)blockIdx.x * kc * wzp
                        : reinterpret_cast<T *>(smem_raw);
    T *ybuf = reinterpret_cast<T *>(smem_raw) + (A.zglobal ? 0 : A.zwords);
    T *mbuf = ybuf + A.ywords;
    T *obuf = mbuf + A.mwords;  // outputs before normalisation (scaled)
    const int zlen = kc * wzp;
    const int mchunks = (A.a_leaf || A.defer) ? 0 : (A.Wa * (int)sizeof(T) + 15) / 16;
    const int nvec = (A.Wz + V::n - 1) / V::n;
    // column passes: the CTA's tile covers kWideThreads * NV vectors of the
    // row; wider rows walk their arcs once per tile
    const int npass = A.npass > 0 ? A.npass : 1;
    unsigned ovf = 0;
    for (int64_t ti = blockIdx.x; ti < A.ntasks; ti += gridDim.x) {
        const int4 task = A.tasks[ti];
        const int v = task.x, slot = task.y;
        const int64_t e0 = task.z, e1 = task.w;
        for (int b = 0; b < A.nb; ++b) {
            const int64_t rowb = (int64_t)v * A.nb + b;
            const int cv = A.colours[(int64_t)b * A.n + v];
            const bool cok = (unsigned)cv < (unsigned)kc && e0 < e1;
            const int eref = SCALED ? row_eref(A, rowb) : 0;
            if (mchunks && cok) {
                const char *src = static_cast<const char *>(A.Ma) + rowb * A.lda * sizeof(T);
                for (int c = tid; c < mchunks; c += blockDim.x) {
                    const unsigned dst = (unsigned)__cvta_generic_to_shared(reinterpret_cast<char *>(mbuf) + 16 * c);
                    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(dst), "l"(src + 16 * c) : "memory");
                }
                asm volatile("cp.async.commit_group;\n" ::: "memory");
            }
            for (int pass = 0; cok && pass < npass; ++pass) {
                const int vbase = pass * kWideThreads * NV + w * 32 * NV + lane;  // this lane's first vector
                bool qok[NV];
#pragma unroll
                for (int q = 0; q < NV; ++q) qok[q] = vbase + 32 * q < nvec;
                // integer tables of odd width: the last vector's padding element is cleared
                bool tail[NV];
#pragma unroll
                for (int q = 0; q < NV; ++q)
                    tail[q] = Ar<T>::exact && V::n == 2 && (A.Wz & 1) && vbase + 32 * q == nvec - 1;
                // sum colour runs of the arcs into this warp's slice of Z: each
                // colour's slice is written once; colours without arcs are
                // zeroed after the walk (v's own colour is read by nothing)
                const int64_t uvec = (int64_t)A.nb * A.ldp / V::n;
                const VT *Mb = reinterpret_cast<const VT *>(static_cast<const T *>(A.Mp) + (int64_t)b * A.ldp) + vbase;
                const int32_t *scol = A.scol + (int64_t)b * A.nnz;
                const int8_t *sclr = A.sclr + (int64_t)b * A.nnz;
                const float *sw = WEIGHTED ? A.sw + (int64_t)b * A.nnz : nullptr;
                const int16_t *Ep = SCALED ? A.Ep + b : nullptr;
                VT run[NV];
#pragma unroll
                for (int q = 0; q < NV; ++q) run[q] = V::zero();
                int cur = -1;
                uint32_t seen = 0;
                auto flush = [&](int c) {
                    if (c != cv) {
                        VT *zr = reinterpret_cast<VT *>(zbuf + c * wzp) + vbase;
#pragma unroll
                        for (int q = 0; q < NV; ++q)
                            if (qok[q]) zr[32 * q] = run[q];
                        seen |= 1u << c;
                    }
#pragma unroll
                    for (int q = 0; q < NV; ++q) run[q] = V::zero();
                };
                // slots past the live arcs read the zero row (vertex n)
                const int zero_row = (int)A.n;
                for (int64_t base = e0; base < e1; base += 32) {
                    const int cnt_in = (int)(e1 - base < 32 ? e1 - base : 32);
                    const int c_in = lane < cnt_in ? (int)__ldg(sclr + base + lane) : -1;
                    const bool t_in = c_in >= 0 && c_in != cv;
                    const int u_in = t_in ? __ldg(scol + base + lane) : zero_row;
                    // compacted to the arcs that add something, as in spmm_z
                    const unsigned live_in = __ballot_sync(kFull, t_in);
                    const int cnt = __popc(live_in);
                    const bool t_l = lane < cnt;
                    const int src = t_l ? (int)__fns(live_in, 0, lane + 1) : lane;
                    int u_l = __shfl_sync(kFull, u_in, src);
                    int c_l = __shfl_sync(kFull, c_in, src);
                    const int c_last = __shfl_sync(kFull, c_l, cnt > 0 ? cnt - 1 : 0);
                    if (!t_l) {
                        u_l = zero_row;
                        c_l = c_last;
                    }
                    T w_l = T(1);
                    if (WEIGHTED) w_l = t_l ? T(__ldg(sw + base + src)) : T(0);
                    int ep_l = eref;
                    if (SCALED && t_l) ep_l = (int)__ldg(Ep + (int64_t)u_l * A.nb);
                    for (int j0 = 0; j0 < cnt; j0 += U) {
                        VT x[U][NV];
                        T wr[U];
                        int cr[U];
#pragma unroll
                        for (int r = 0; r < U; ++r) {
                            const int j = j0 + r;
                            const int u = __shfl_sync(kFull, u_l, j);
                            cr[r] = __shfl_sync(kFull, c_l, j);
                            wr[r] = WEIGHTED ? __shfl_sync(kFull, w_l, j) : T(1);
                            if (SCALED) {
                                const int ep = __shfl_sync(kFull, ep_l, j);
                                wr[r] *= T(exp2_neg(ep - eref));
                            }
                            const VT *row = Mb + (int64_t)u * uvec;
#pragma unroll
                            for (int q = 0; q < NV; ++q) {
                                // FP32 loads of the first tile are unpredicated (the
                                // table's padding covers a tile past its last row)
                                x[r][q] = ((sizeof(T) == 4 && pass == 0 && !A.pred_lanes) || qok[q]) ? ldg_row(row + 32 * q)
                                                                                    : V::zero();
                                if constexpr (Ar<T>::exact && V::n == 2)
                                    if (tail[q]) x[r][q].y = 0;
                            }
                        }
#pragma unroll
                        for (int r = 0; r < U; ++r) {
                            if (cr[r] != cur) {
                                if (cur >= 0) flush(cur);
                                cur = cr[r];
                            }
#pragma unroll
                            for (int q = 0; q < NV; ++q) {
                                if (FMA)
                                    V::fma(run[q], wr[r], x[r][q]);
                                else
                                    vadd<T>(run[q], x[r][q], ovf);
                            }
                        }
                    }
                }
                if (cur >= 0) flush(cur);
                for (int d = 0; d < kc; ++d) {
                    if (!(seen >> d & 1u) && d != cv) {
                        VT *zr = reinterpret_cast<VT *>(zbuf + d * wzp) + vbase;
#pragma unroll
                        for (int q = 0; q < NV; ++q)
                            if (qok[q]) zr[32 * q] = V::zero();
                    }
                }
            }
            __syncthreads();
            if (slot >= 0 && cok) {
                T *sc = static_cast<T *>(A.scratch) + ((int64_t)slot * A.nb + b) * A.scratch_ld;
                // (the row of v's own colour in Z is stale and read by nothing)
                for (int j = tid; j < zlen; j += blockDim.x)
                    if (j < cv * wzp || j >= (cv + 1) * wzp) atomic_add(sc + j, zbuf[j], ovf);
                __threadfence();
                __syncthreads();
                if (tid == 0) {
                    const unsigned done = atomicAdd(A.counters + (int64_t)slot * A.nb + b, 1u);
                    s_last = (done + 1u == (unsigned)__ldg(A.heavy_chunks + slot));
                }
                __syncthreads();
                if (!s_last) {
                    if (mchunks) asm volatile("cp.async.wait_all;\n" ::: "memory");
                    __syncthreads();
                    continue;
                }
                __threadfence();
                for (int j = tid; j < zlen; j += blockDim.x) zbuf[j] = __ldcg(sc + j);
                __syncthreads();
            }
            // Y' = expansion of Z over the p-sets without v's colour
            if (cok) {
                const int p = A.p, wy = A.wy;
                if (A.expand32) {
                    // 32-bit offsets (Z of more than 65,536 elements)
                    const uint32_t *ex = A.expand32 + (int64_t)cv * wy * p;
                    for (int j = tid; j < wy; j += blockDim.x) {
                        T s = T(0);
                        for (int k = 0; k < p; ++k) Ar<T>::add(s, zbuf[__ldg(ex + (int64_t)j * p + k)], ovf);
                        ybuf[j] = s;
                    }
                } else {
                    const uint16_t *ex = A.expand + (int64_t)cv * wy * A.pstride;
                    for (int j = tid; j < wy; j += blockDim.x) ybuf[j] = expand_set(ex, A.pstride, p, j, zbuf, ovf);
                }
            }
            if (mchunks && cok) asm volatile("cp.async.wait_all;\n" ::: "memory");
            __syncthreads();
            if (A.Yout && (!SCALED || A.defer)) {
                T *yo = static_cast<T *>(A.Yout) + rowb * A.ldy;
                for (int j = tid; j < A.wy; j += blockDim.x) yo[j] = cok ? ybuf[j] : T(0);
            }
            if (A.defer) {
                // the eMA runs in its own launch over blocks of rows
                __syncthreads();
                continue;
            }
            // eMA in squeezed coordinates over the whole CTA
            const int base = SCALED ? (A.a_leaf ? 0 : (int)A.Ea[rowb]) + eref : 0;
            if (A.root) {
                T sum = group_sum_chk<32>(ema_root_partial<T, kWideThreads>(A, cok, ybuf, mbuf, tid, ovf), ovf);
                if (lane == 0) s_red[w] = sum;
                __syncthreads();
                if (tid == 0) {
                    T t = T(0);
                    for (int i = 0; i < kWideWarps; ++i) Ar<T>::add(t, s_red[i], ovf);
                    if constexpr (SCALED)
                        A.root_out_d[(int64_t)b * A.n + v] = cok ? ldexp((double)t, base) : 0.0;
                    else
                        static_cast<T *>(A.root_out)[(int64_t)b * A.n + v] = t;
                }
            } else if constexpr (SCALED) {
                // outputs to obuf, then the row is normalised by its largest value
                T mx = T(0);
                ema_rows<T, kWideThreads>(A, cok, ybuf, mbuf, tid, ovf, [&](int S, T x) {
                    obuf[S] = x;
                    mx = fmax(mx, x);
                });
                mx = warp_max(mx);
                if (lane == 0) s_max[w] = mx;
                __syncthreads();
                T m = T(0);
                for (int i = 0; i < kWideWarps; ++i) m = fmax(m, s_max[i]);
                const int em = m > T(0) ? ilogb(m) : 0;
                T *out = static_cast<T *>(A.Ms) + rowb * A.ldt;
                for (int j = tid; j < A.Ws; j += blockDim.x) out[j] = ldexp(obuf[j], -em);
                if (tid == 0) A.Es[rowb] = m > T(0) ? clamp_exp(base + em) : kEmptyRowExp;
            } else {
                T *out = static_cast<T *>(A.Ms) + rowb * A.ldt;
                const bool accumulate = A.accumulate != 0;
                ema_rows<T, kWideThreads>(A, cok, ybuf, mbuf, tid, ovf, [&](int S, T x) {
                    if (accumulate) Ar<T>::add(x, out[S], ovf);
                    out[S] = x;
                });
            }
            __syncthreads();
        }
        report_ovf<T>(A.status, ovf);
    }
}

template <typename T, int G, int NV, bool HIST, bool WEIGHTED, bool SC, int FORM = 0>
void *kernel_ptr() {
    return reinterpret_cast<void *>(&node_kernel<T, G, NV, HIST, WEIGHTED, SC, FORM>);
}

template <typename T, bool W, bool SC = false>
void *pick(bool hist, int g, int nv, int form = 0) {
    if (hist) return kernel_ptr<T, 32, 1, true, W, SC>();
    if constexpr (!SC && !std::is_same<T, u128>::value) {
        if (g == 32 && form == 1) return nv == 1 ? kernel_ptr<T, 32, 1, false, W, SC, 1>()
                                                 : kernel_ptr<T, 32, 2, false, W, SC, 1>();
        if (g == 32 && form == 2) return nv == 1 ? kernel_ptr<T, 32, 1, false, W, SC, 2>()
                                                 : kernel_ptr<T, 32, 2, false, W, SC, 2>();
    }
    if (g == 4) return kernel_ptr<T, 4, 1, false, W, SC>();
    if (g == 8) return kernel_ptr<T, 8, 1, false, W, SC>();
    if (g == 16) return kernel_ptr<T, 16, 1, false, W, SC>();
    switch (nv) {
        case 1: return kernel_ptr<T, 32, 1, false, W, SC>();
        case 2: return kernel_ptr<T, 32, 2, false, W, SC>();
        case 3: return kernel_ptr<T, 32, 3, false, W, SC>();
        case 4: return kernel_ptr<T, 32, 4, false, W, SC>();
        default: return nullptr;
    }
}

template <typename T, bool W, bool SC = false>
void *pick_wide(int nv) {
    switch (nv) {
        case 1: return reinterpret_cast<void *>(&node_wide_kernel<T, 1, W, SC>);
        case 2: return reinterpret_cast<void *>(&node_wide_kernel<T, 2, W, SC>);
        case 3: return reinterpret_cast<void *>(&node_wide_kernel<T, 3, W, SC>);
        case 4: return reinterpret_cast<void *>(&node_wide_kernel<T, 4, W, SC>);
        default: return nullptr;
    }
}

template <typename T, bool W, bool SC>
void *pick_group(int g, int form = 0) {
    if constexpr (!SC && !std::is_same<T, u128>::value) {
        if (form == 1) {
            if (g == 4) return reinterpret_cast<void *>(&node_group_kernel<T, 4, W, SC, 1>);
            if (g == 8) return reinterpret_cast<void *>(&node_group_kernel<T, 8, W, SC, 1>);
            if (g == 16) return reinterpret_cast<void *>(&node_group_kernel<T, 16, W, SC, 1>);
            return nullptr;
        }
    }
    if (g == 4) return reinterpret_cast<void *>(&node_group_kernel<T, 4, W, SC>);
    if (g == 8) return reinterpret_cast<void *>(&node_group_kernel<T, 8, W, SC>);
    if (g == 16) return reinterpret_cast<void *>(&node_group_kernel<T, 16, W, SC>);
    return nullptr;
}

void *select_kernel(Elem e, bool hist, int g, int nv, bool weighted, bool group = false, int form = 0) {
    // integer tables count unweighted graphs only
    if ((e == Elem::U64 || e == Elem::U128) && weighted) return nullptr;
    if (group) {
        if (hist || nv != 1) return nullptr;
        if (e == Elem::U64) return pick_group<u64, false, false>(g, form);
        if (e == Elem::U128) return pick_group<u128, false, false>(g);
        if (e == Elem::F64)
            return weighted ? pick_group<double, true, false>(g, form) : pick_group<double, false, false>(g, form);
        return weighted ? pick_group<float, true, false>(g, form) : pick_group<float, false, false>(g, form);
    }
    if (g == kWideLanes) {
        // wide rows: one CTA per task (nv vectors per lane, 8 warps)
        if (hist) return nullptr;
        if (e == Elem::U64) return pick_wide<u64, false>(nv);
        if (e == Elem::U128) return pick_wide<u128, false>(nv);
        if (e == Elem::F64) return weighted ? pick_wide<double, true>(nv) : pick_wide<double, false>(nv);
        return weighted ? pick_wide<float, true>(nv) : pick_wide<float, false>(nv);
    }
    if (e == Elem::U64) return pick<u64, false>(hist, g, nv, form);
    if (e == Elem::U128) return pick<u128, false>(hist, g, nv);
    if (e == Elem::F64) return weighted ? pick<double, true>(hist, g, nv, form) : pick<double, false>(hist, g, nv, form);
    return weighted ? pick<float, true>(hist, g, nv, form) : pick<float, false>(hist, g, nv, form);
}

void *select_kernel_scaled(bool hist, int g, int nv, bool weighted, bool group = false) {
    if (group) {
        if (hist || nv != 1) return nullptr;
        return weighted ? pick_group<float, true, true>(g) : pick_group<float, false, true>(g);
    }
    if (g == kWideLanes) {
        if (hist) return nullptr;
        return weighted ? pick_wide<float, true, true>(nv) : pick_wide<float, false, true>(nv);
    }
    return weighted ? pick<float, true, true>(hist, g, nv) : pick<float, false, true>(hist, g, nv);
}

// ------------------------------------------------------------- reductions

__device__ __forceinline__ void two_sum(double a, double b, double &s, double &e) {
    s = a + b;
    const double bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

__device__ __forceinline__ void rs_combine(RootSum &x, const RootSum &y) {
    const unsigned long long lo = x.lo + y.lo;
    const unsigned long long hi = x.hi + y.hi + (lo < x.lo ? 1ull : 0ull);
    if (hi < x.hi || (hi == x.hi && y.hi + (lo < x.lo ? 1ull : 0ull) != 0ull)) x.flags |= kFlagNotIntegral;  // 2^128 wrap
    x.hi = hi;
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
__global__ void root_partial_kernel(const T *vals, int64_t n, int64_t live, double *pv, const int32_t *pvmap,
                                    RootSum *partials, int chunks) {
    __shared__ RootSum red[32];
    const int seg = blockIdx.y;
    const int chunk = blockIdx.x;
    const int64_t per = (n + chunks - 1) / chunks;
    const int64_t lo = (int64_t)chunk * per;
    const int64_t hi_all = (lo + per < n) ? lo + per : n;
    // entries past `live` are zeros (isolated vertices): not read
    const int64_t hi = hi_all < live ? hi_all : live;
    if (pv)
        for (int64_t i = (lo > live ? lo : live) + threadIdx.x; i < hi_all; i += blockDim.x)
            pv[(int64_t)seg * n + (pvmap ? (int64_t)pvmap[i] : i)] = 0.0;
    RootSum acc = rs_from(0.0);
    if constexpr (sizeof(T) == 4) {
        // FP32 tables: the exact integer path buys nothing; each thread sums
        // in double (the per-thread sums are then combined compensated)
        double sum = 0.0;
        unsigned bad = 0;
        const T *sv = vals + (int64_t)seg * n;
        if (pv) {
            for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) {
                const T x = sv[i];
                pv[(int64_t)seg * n + (pvmap ? (int64_t)pvmap[i] : i)] = (double)x;
                if (isfinite(x))
                    sum += (double)x;
                else
                    bad = 1;
            }
        } else {
            // four loads in flight per thread
            const int64_t step = blockDim.x;
            int64_t i = lo + threadIdx.x;
            for (; i + 3 * step < hi; i += 4 * step) {
                const T x0 = sv[i], x1 = sv[i + step], x2 = sv[i + 2 * step], x3 = sv[i + 3 * step];
                bad |= !isfinite(x0) | !isfinite(x1) | !isfinite(x2) | !isfinite(x3);
                sum += ((double)x0 + (double)x1) + ((double)x2 + (double)x3);
            }
            for (; i < hi; i += step) {
                const T x = sv[i];
                bad |= !isfinite(x);
                sum += (double)x;
            }
            if (bad) sum = 0.0;
        }
        acc.s = sum;
        acc.flags = kFlagNotIntegral | (bad ? kFlagNonFinite : 0u);
    } else if constexpr (Ar<T>::exact) {
        // integer tables: the 128-bit sum directly (and a double sum beside it)
        for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) {
            const T x = vals[(int64_t)seg * n + i];
            RootSum r = rs_from(0.0);
            if constexpr (std::is_same<T, u128>::value) {
                r.lo = x.lo;
                r.hi = x.hi;
                r.s = u128_to_double(x.hi, x.lo);
            } else {
                r.lo = x;
                r.s = __ull2double_rn(x);
            }
            if (pv) pv[(int64_t)seg * n + (pvmap ? (int64_t)pvmap[i] : i)] = r.s;
            rs_combine(acc, r);
        }
    } else {
        for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) {
            const double v = (double)vals[(int64_t)seg * n + i];
            if (pv) pv[(int64_t)seg * n + (pvmap ? (int64_t)pvmap[i] : i)] = v;
            rs_combine(acc, rs_from(v));
        }
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

// One block per segment: each thread combines a strided share of the
// segment's partials, then the block combines its threads' results (the
// 128-bit integer sum is exact in any order).
__global__ void __launch_bounds__(256) root_final_kernel(const RootSum *partials, int chunks, int nseg,
                                                         RootSum *out) {
    __shared__ RootSum red[8];
    const int seg = blockIdx.x;
    if (seg >= nseg) return;
    RootSum t = rs_from(0.0);
    for (int i = threadIdx.x; i < chunks; i += blockDim.x) rs_combine(t, partials[(int64_t)seg * chunks + i]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const RootSum y = rs_shfl_xor(t, o);
        rs_combine(t, y);
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) red[w] = t;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int i = 1; i < (int)(blockDim.x >> 5); ++i) rs_combine(t, red[i]);
        out[seg] = t;
    }
}

// Reference exponent of each row for the scaled FP32 gather: the largest
// exponent among the passive rows it will add up (arcs to neighbours of a
// valid colour other than its own), one warp per (task, colouring).  Split
// rows combine their chunks with atomicMax; Eref is pre-filled below -2^15.
__global__ void eref_kernel(const int4 *__restrict__ tasks, int64_t ntasks, const int32_t *__restrict__ scol,
                            const int8_t *__restrict__ sclr, const int8_t *__restrict__ colours, int64_t n,
                            int64_t nnz, int nb, int kc, const int16_t *__restrict__ Ep, int32_t *Eref) {
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t items = ntasks * nb;
    for (int64_t it = (((int64_t)blockIdx.x * blockDim.x) >> 5) + (threadIdx.x >> 5); it < items; it += nwarps) {
        const int64_t ti = it / nb;
        const int b = (int)(it - ti * nb);
        const int4 task = tasks[ti];
        const int cv = colours[(int64_t)b * n + task.x];
        int m = kEmptyRowExp;
        for (int64_t e = task.z + lane; e < task.w; e += 32) {
            const int c = sclr[(int64_t)b * nnz + e];
            if (c >= 0 && c != cv) {
                const int u = scol[(int64_t)b * nnz + e];
                const int x = Ep[(int64_t)u * nb + b];
                m = x > m ? x : m;
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const int y = __shfl_xor_sync(kFull, m, o);
            m = y > m ? y : m;
        }
        if (lane == 0 && (unsigned)cv < (unsigned)kc) atomicMax(Eref + (int64_t)task.x * nb + b, m);
    }
}

// Entry j of row `row` of a fused histogram table: cnt neighbours (added
// atomically for chunks of split rows).
__device__ __forceinline__ void hist_put(const SortHist &H, int64_t row, int j, unsigned cnt, bool atomic) {
    const int64_t at = row * H.ld + j;
    switch (H.elem) {
        case Elem::F32: {
            float *p = static_cast<float *>(H.out) + at;
            if (!atomic)
                *p = (float)cnt;
            else if (cnt)
                atomicAdd(p, (float)cnt);
            break;
        }
        case Elem::F64: {
            double *p = static_cast<double *>(H.out) + at;
            if (!atomic)
                *p = (double)cnt;
            else if (cnt)
                atomicAdd(p, (double)cnt);
            break;
        }
        case Elem::U64: {
            u64 *p = static_cast<u64 *>(H.out) + at;
            if (!atomic)
                *p = cnt;
            else if (cnt)
                atomicAdd(p, (u64)cnt);
            break;
        }
        default: {
            u128 *p = static_cast<u128 *>(H.out) + at;
            if (!atomic)
                *p = u128((u64)cnt, 0ull);
            else if (cnt)
                atomicAdd(&p->lo, (u64)cnt);  // counts stay far below 2^64
            break;
        }
    }
}

// The fused histogram row of (task, b) from per-colour counts cnt(x) (x in
// [0, kc)): lane j < kc - 1 writes the count of the j-th colour other than cv.
template <typename F>
__device__ __forceinline__ void hist_row(const SortHist &H, const int4 &task, int b, int nb, int cv, int kc, int j,
                                         F &&cnt) {
    const int64_t row = (int64_t)task.x * nb + b;
    if (H.hcount && j < kc) {
        // the full count row (invalid colours of v included: the nodes check it)
        int32_t *p = H.hcount + row * H.hld + j;
        const int c = (int)cnt(j);
        if (task.y < 0)
            *p = c;
        else if (c)
            atomicAdd(p, c);
    }
    if (!H.out || j >= kc - 1) return;
    const bool ok = (unsigned)cv < (unsigned)kc;
    const int x = j < cv ? j : j + 1;
    hist_put(H, row, j, ok ? (unsigned)cnt(x) : 0u, task.y >= 0);
}

// The same sort for tasks of at most G arcs, 32 / G tasks per warp: a lane's
// arc goes to the number of the task's arcs with a smaller colour (or the
// same colour and a lower index), counted over the group with shuffles.
template <int G>
__global__ void colour_sort_small_kernel(const int4 *__restrict__ tasks, int64_t ntasks,
                                         const int32_t *__restrict__ col_idx, const float *__restrict__ weights,
                                         int64_t n, int64_t nnz, const int8_t *__restrict__ colours, int nb, int kc,
                                         int32_t *scol, int8_t *sclr, float *sw, const SortHist H) {
    constexpr int NG = 32 / G;
    const int lane = threadIdx.x & 31, grp = lane / G, gl = lane % G, g0 = grp * G;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t rounds = (ntasks + NG - 1) / NG;
    for (int64_t rd = (((int64_t)blockIdx.x * blockDim.x) >> 5) + (threadIdx.x >> 5); rd < rounds; rd += nwarps) {
        const int64_t t = rd * NG + grp;
        const int4 task = t < ntasks ? tasks[t] : make_int4(0, -1, 0, 0);
        const int m = task.w - task.z;  // at most G
        const bool in = gl < m;
        const int u = in ? __ldg(col_idx + task.z + gl) : 0;
        for (int b = 0; b < nb; ++b) {
            int c = in ? (int)__ldg(colours + (int64_t)b * n + u) : 0x7fff;
            if (in && (unsigned)c >= (unsigned)kc) c = kc;  // invalid colours last
            int rank = 0;
#pragma unroll
            for (int k = 0; k < G; ++k) {
                const int ck = __shfl_sync(kFull, c, g0 + k);
                rank += (k < m) && (ck < c || (ck == c && k < gl));
            }
            if (in) {
                const int64_t pos = (int64_t)b * nnz + task.z + rank;
                scol[pos] = u;
                if (H.perm) H.perm[pos] = task.z + gl;
                sclr[pos] = (int8_t)(c == kc ? -1 : c);
                if (sw) sw[pos] = __ldg(weights + task.z + gl);
            }
            if (H.out || H.hcount) {
                // lane gl counts colours gl and gl + G of its task's arcs
                unsigned n0 = 0, n1 = 0;
#pragma unroll
                for (int k = 0; k < G; ++k) {
                    const int ck = __shfl_sync(kFull, c, g0 + k);
                    n0 += (k < m) && ck == gl;
                    n1 += (k < m) && ck == gl + G;
                }
                const bool have = t < ntasks;
                const int cv = have ? (int)__ldg(colours + (int64_t)b * n + task.x) : -1;
                // the count of colour x lives on lane x % G of the group (n0 or n1)
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int j = gl + G * h;  // output entry j: colour j or j + 1
                    const int x = j < cv ? j : j + 1;
                    const unsigned c0 = __shfl_sync(kFull, n0, g0 + (x % G));
                    const unsigned c1 = __shfl_sync(kFull, n1, g0 + (x % G));
                    if (have && H.out) {
                        SortHist Ho = H;
                        Ho.hcount = nullptr;
                        hist_row(Ho, task, b, nb, cv, kc, j, [&](int) { return x < G ? c0 : c1; });
                    }
                    // the full count row: colour j is this lane's own count
                    if (have && H.hcount && j < kc) {
                        int32_t *p = H.hcount + ((int64_t)task.x * nb + b) * H.hld + j;
                        const int cj = (int)(h == 0 ? n0 : n1);
                        if (task.y < 0)
                            *p = cj;
                        else if (cj)
                            atomicAdd(p, cj);
                    }
                }
            }
        }
    }
}

// Stable counting sort by neighbour colour of the arcs of each work-list task
// (a row, or a chunk of a split row), one warp per task for every colouring
// of the wave; colours outside [0, kc) go last, tagged -1.  Each colour then
// forms one run per task.  Tasks of at most 32 arcs sort in one pass from
// registers; longer ones count buckets first, then place.
constexpr int kSortStage = 1024;

// HIST: some histogram output is requested (H.out or H.hcount); without it
// the kernel carries none of that code.
template <bool HIST>
__global__ void colour_sort_kernel(const int4 *__restrict__ tasks, int64_t ntasks, const int32_t *__restrict__ col_idx,
                                   const float *__restrict__ weights, int64_t n, int64_t nnz,
                                   const int8_t *__restrict__ colours, int nb, int kc, int32_t *scol, int8_t *sclr,
                                   float *sw, const SortHist H) {
    __shared__ int base_s[8][kMaxHistColours + 1];
    // tasks of up to kSortStage arcs keep their neighbours and colours here
    // between the counting pass and the placing pass
    __shared__ int32_t ubuf_s[8][kSortStage];
    __shared__ int8_t cbuf_s[8][kSortStage];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    int *start = base_s[wib];
    int32_t *ubuf = ubuf_s[wib];
    int8_t *cbuf = cbuf_s[wib];
    const unsigned lt = (1u << lane) - 1u;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    // software pipeline over the warp's tasks: the descriptor two tasks ahead
    // and the neighbours of the next task (when it has at most 32 arcs) load
    // while the current task sorts
    int64_t t = (((int64_t)blockIdx.x * blockDim.x) >> 5) + wib;
    const int4 none = make_int4(0, -1, 0, 0);
    int4 task = t < ntasks ? tasks[t] : none;
    int4 next = t + nwarps < ntasks ? tasks[t + nwarps] : none;
    int u_cur = task.w - task.z <= 32 && task.z + lane < task.w ? __ldg(col_idx + task.z + lane) : 0;
    for (; t < ntasks; t += nwarps) {
        const int4 after = t + 2 * nwarps < ntasks ? tasks[t + 2 * nwarps] : none;
        const int u_next = next.w - next.z <= 32 && next.z + lane < next.w ? __ldg(col_idx + next.z + lane) : 0;
        const int64_t e0 = task.z, e1 = task.w;
        const bool single = e1 - e0 <= 32;
        // a task of at most 32 arcs keeps its neighbours in registers
        const int64_t e_one = e0 + lane;
        const int u_one = u_cur;
        for (int b = 0; b < nb; ++b) {
            const int8_t *col = colours + (int64_t)b * n;
            int32_t *so = scol + (int64_t)b * nnz + e0;
            int8_t *co = sclr + (int64_t)b * nnz + e0;
            float *wo = sw ? sw + (int64_t)b * nnz + e0 : nullptr;
            int32_t *po = H.perm ? H.perm + (int64_t)b * nnz + e0 : nullptr;
            if (single) {
                // one batch: bucket sizes from the groups of equal colours
                const bool ok = e_one < e1;
                int c = ok ? (int)__ldg(col + u_one) : -2;
                if (ok && (unsigned)c >= (unsigned)kc) c = kc;  // bucket kc holds invalid colours
                const unsigned same = __match_any_sync(kFull, c);
                if (lane <= kc) start[lane] = 0;
                __syncwarp();
                if (ok && (same & lt) == 0) start[c] = __popc(same);
                __syncwarp();
                if (HIST)
                    hist_row(H, task, b, nb, (int)__ldg(col + task.x), kc, lane, [&](int x) { return start[x]; });
                const int cnt = lane <= kc ? start[lane] : 0;
                int incl = cnt;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int y = __shfl_up_sync(kFull, incl, o);
                    if (lane >= o) incl += y;
                }
                __syncwarp();
                if (lane <= kc) start[lane] = incl - cnt;
                __syncwarp();
                if (ok) {
                    const int pos = start[c] + __popc(same & lt);
                    so[pos] = u_one;
                    co[pos] = (int8_t)(c == kc ? -1 : c);
                    if (wo) wo[pos] = __ldg(weights + e_one);
                    if (po) po[pos] = (int32_t)e_one;
                }
                __syncwarp();
                continue;
            }
            // pass 1: arcs per colour (bucket kc holds invalid colours)
            if (lane <= kc) start[lane] = 0;
            __syncwarp();
            if (e1 - e0 <= kSortStage) {
                // four batches of neighbours, then their colours, load together;
                // both are staged for the placing pass
                for (int64_t e = e0 + lane; e - lane < e1; e += 128) {
                    int uu[4], cc[4];
#pragma unroll
                    for (int k = 0; k < 4; ++k) uu[k] = e + 32 * k < e1 ? __ldg(col_idx + e + 32 * k) : 0;
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        const bool ok = e + 32 * k < e1;
                        cc[k] = ok ? (int)__ldg(col + uu[k]) : -2;
                        if (ok && (unsigned)cc[k] >= (unsigned)kc) cc[k] = kc;
                    }
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        const int64_t ek = e + 32 * k;
                        if (ek - lane >= e1) break;  // warp-uniform: no such batch
                        const bool ok = ek < e1;
                        const unsigned same = __match_any_sync(kFull, cc[k]);
                        if (ok) {
                            ubuf[ek - e0] = uu[k];
                            cbuf[ek - e0] = (int8_t)cc[k];
                            if ((same & lt) == 0) start[cc[k]] += __popc(same);
                        }
                        __syncwarp();
                    }
                }
                if (HIST)
                    hist_row(H, task, b, nb, (int)__ldg(col + task.x), kc, lane, [&](int x) { return start[x]; });
                const int cnt = lane <= kc ? start[lane] : 0;
                int incl = cnt;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int y = __shfl_up_sync(kFull, incl, o);
                    if (lane >= o) incl += y;
                }
                __syncwarp();
                if (lane <= kc) start[lane] = incl - cnt;
                __syncwarp();
                // pass 2 from the staged copies
                for (int64_t e = e0 + lane; e - lane < e1; e += 32) {
                    const bool ok = e < e1;
                    const int u = ok ? ubuf[e - e0] : 0;
                    const int c = ok ? (int)cbuf[e - e0] : -2;
                    const unsigned same = __match_any_sync(kFull, c);
                    if (ok) {
                        const int pos = start[c] + __popc(same & lt);
                        so[pos] = u;
                        co[pos] = (int8_t)(c == kc ? -1 : c);
                        if (wo) wo[pos] = __ldg(weights + e);
                        if (po) po[pos] = (int32_t)e;
                    }
                    __syncwarp();
                    if (ok && (same & lt) == 0) start[c] += __popc(same);
                    __syncwarp();
                }
                continue;
            }
            for (int64_t e = e0 + lane; e - lane < e1; e += 32) {
                const bool ok = e < e1;
                int c = ok ? (int)__ldg(col + __ldg(col_idx + e)) : -2;
                if (ok && (unsigned)c >= (unsigned)kc) c = kc;
                const unsigned same = __match_any_sync(kFull, c);
                if (ok && (same & lt) == 0) start[c] += __popc(same);
                __syncwarp();
            }
            if (HIST)
                hist_row(H, task, b, nb, (int)__ldg(col + task.x), kc, lane, [&](int x) { return start[x]; });
            // exclusive prefix over buckets
            const int cnt = lane <= kc ? start[lane] : 0;
            int incl = cnt;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(kFull, incl, o);
                if (lane >= o) incl += y;
            }
            __syncwarp();
            if (lane <= kc) start[lane] = incl - cnt;
            __syncwarp();
            // pass 2: stable placement
            for (int64_t e = e0 + lane; e - lane < e1; e += 32) {
                const bool ok = e < e1;
                const int u = ok ? __ldg(col_idx + e) : 0;
                int c = ok ? (int)__ldg(col + u) : -2;
                if (ok && (unsigned)c >= (unsigned)kc) c = kc;
                const unsigned same = __match_any_sync(kFull, c);
                if (ok) {
                    const int pos = start[c] + __popc(same & lt);
                    so[pos] = u;
                    co[pos] = (int8_t)(c == kc ? -1 : c);
                    if (wo) wo[pos] = __ldg(weights + e);
                    if (po) po[pos] = (int32_t)e;
                }
                __syncwarp();
                // advance every bucket by its arcs in this batch (leader lane of each group)
                if (ok && (same & lt) == 0) start[c] += __popc(same);
                __syncwarp();
            }
        }
        task = next;
        next = after;
        u_cur = u_next;
    }
}

// ---------------------------------------------------------------- backward

template <typename T>
__global__ void bwd_ema_kernel(const BwdEmaArgs A) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int per = A.ws + A.wa + A.wy;
    T *gs = reinterpret_cast<T *>(smem_raw) + (int64_t)wib * per;
    T *ma = gs + A.ws;
    T *yy = ma + A.wa;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t v = (((int64_t)blockIdx.x * blockDim.x) >> 5) + wib; v < A.n; v += nwarps) {
        const int c = A.colours[v];
        T *yb = static_cast<T *>(A.Ybar) + v * A.ldyb;
        if ((unsigned)c >= (unsigned)A.kc) {
            for (int j = lane; j < A.wy; j += 32) yb[j] = T(0);
            continue;
        }
        const T seed = A.seed ? T(A.seed[v]) : T(0);
        const T *g = A.G ? static_cast<const T *>(A.G) + v * A.ldg : nullptr;
        for (int j = lane; j < A.ws; j += 32) gs[j] = g ? g[j] : seed;
        if (A.a >= 2) {
            const T *mr = static_cast<const T *>(A.Ma) + v * A.lda;
            const T *yr = static_cast<const T *>(A.Y) + v * A.ldy;
            for (int j = lane; j < A.wa; j += 32) ma[j] = mr[j];
            for (int j = lane; j < A.wy; j += 32) yy[j] = yr[j];
        }
        __syncwarp();
        if (A.a == 1) {
            for (int j = lane; j < A.wy; j += 32) yb[j] = gs[j];
        } else {
            for (int j = lane; j < A.wy; j += 32) {
                const uint32_t *pr = A.ybar + (int64_t)j * A.nybar;
                T acc = T(0);
                for (int i = 0; i < A.nybar; ++i) {
                    const uint32_t x = __ldg(pr + i);
                    acc = fma(gs[x & 0xffffu], ma[x >> 16], acc);
                }
                yb[j] = acc;
            }
            T *ga = static_cast<T *>(A.Gabar) + v * A.ldga;
            for (int j = lane; j < A.wa; j += 32) {
                const uint32_t *pr = A.mabar + (int64_t)j * A.nmabar;
                T acc = T(0);
                for (int i = 0; i < A.nmabar; ++i) {
                    const uint32_t x = __ldg(pr + i);
                    acc = fma(gs[x & 0xffffu], yy[x >> 16], acc);
                }
                ga[j] += acc;
            }
        }
        __syncwarp();
    }
}

// Per-arc weight gradient, one warp per unit of work: a work-list task (a
// row, or a chunk of at most a chunk's arcs of a long row) when A.tasks is
// set, else a whole row.  Each arc's gradient is its own output, so the
// chunks of a split row need no combining; hub rows cut into chunks keep one
// warp from walking tens of thousands of arcs alone.
template <typename T>
__global__ void sddmm_kernel(const SddmmArgs A) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    T *mp = reinterpret_cast<T *>(smem_raw) + (int64_t)wib * ((A.wmp + 3) / 4 * 4);
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t units = A.tasks ? A.ntasks : A.n;
    for (int64_t t = (((int64_t)blockIdx.x * blockDim.x) >> 5) + wib; t < units; t += nwarps) {
        int64_t u, e0, e1;
        if (A.tasks) {
            const int4 task = A.tasks[t];
            u = task.x;
            e0 = task.z;
            e1 = task.w;
        } else {
            u = t;
            e0 = A.row_ptr[u];
            e1 = A.row_ptr[u + 1];
        }
        if (e0 == e1) continue;
        const int cu = A.colours[u];
        if ((unsigned)cu >= (unsigned)A.kc) continue;
        if (!A.hist) {
            const T *mr = static_cast<const T *>(A.Mp) + u * A.ldp;
            for (int j = lane; j < A.wmp; j += 32) mp[j] = mr[j];
        }
        __syncwarp();
        for (int64_t e = e0 + lane; e < e1; e += 32) {
            const int v = __ldg(A.col_idx + e);
            const int cv = A.colours[v];
            if ((unsigned)cv >= (unsigned)A.kc || cv == cu) continue;
            const uint32_t *pr = A.arc + ((int64_t)cv * A.kc + cu) * A.narc;
            const T *yr = static_cast<const T *>(A.Ybar) + (int64_t)v * A.ldyb;
            T acc = T(0);
            for (int i = 0; i < A.narc; ++i) {
                const uint32_t x = __ldg(pr + i);
                acc = A.hist ? acc + yr[x & 0xffffu] : fma(yr[x & 0xffffu], mp[x >> 16], acc);
            }
            // each arc's slot gains one term per launch: a reduction nothing waits on
            atomicAdd(A.grad + e, (double)acc);
        }
        __syncwarp();
    }
}

// Per-arc weight gradient, row-oriented (p >= 2): for a row v, Zbar(d, i)
// holds Ybar'(v, P) for the p-set P = {d} + (the i-th (p-1)-set of d's
// squeezed universe) when P does not hold v's colour, else 0; then the
// gradient of arc (v, u) is the dot product of Zbar(col(u), .) with the
// compressed row M_p'(u, .).  Groups of G lanes take one arc each (as the
// forward gather does), rows of M_p' are read whole and coalesced, and a
// group's dot product is reduced with shuffles.  One warp per work-list
// task; Zbar in shared memory ([kc][wz_pad] per warp).
template <typename T, int G, int NV>
__global__ void __launch_bounds__(256) sddmm_rows_kernel(const SddmmArgs A) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    using V = Vec16<T>;
    using VT = typename V::type;
    constexpr int NG = 32 / G;
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int grp = lane / G, gl = lane % G;
    const int kc = A.kc, wzp = A.wz_pad;
    T *zb = reinterpret_cast<T *>(smem_raw) + (int64_t)wib * kc * wzp;
    // elements of this lane's vectors inside the row (the row padding past
    // wmp is never written, and 0 times its contents need not be 0)
    int lim[NV];
#pragma unroll
    for (int q = 0; q < NV; ++q) {
        const int left = A.wmp - (gl + G * q) * V::n;
        lim[q] = left < 0 ? 0 : (left > V::n ? V::n : left);
    }
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t ti = (((int64_t)blockIdx.x * blockDim.x) >> 5) + wib; ti < A.ntasks; ti += nwarps) {
        const int4 task = A.tasks[ti];
        const int v = task.x;
        const int cv = A.colours[v];
        if ((unsigned)cv >= (unsigned)kc || task.z == task.w) continue;
        // Zbar of row v
        for (int i = lane; i < kc * wzp; i += 32) zb[i] = T(0);
        __syncwarp();
        const T *yr = static_cast<const T *>(A.Ybar) + (int64_t)v * A.ldyb;
        for (int d = 0; d < kc; ++d) {
            if (d == cv) continue;
            const uint32_t *pr = A.arc + ((int64_t)cv * kc + d) * A.narc;
            for (int k = lane; k < A.narc; k += 32) {
                const uint32_t x = __ldg(pr + k);
                zb[d * wzp + (x >> 16)] = yr[x & 0xffffu];
            }
        }
        __syncwarp();
        for (int64_t base = task.z; base < task.w; base += 32) {
            const int cnt_in = (int)(task.w - base < 32 ? task.w - base : 32);
            const int u_in = lane < cnt_in ? __ldg(A.col_idx + base + lane) : 0;
            const int c_in = lane < cnt_in ? (int)A.colours[u_in] : -1;
            const bool t_in = (unsigned)c_in < (unsigned)kc && c_in != cv;
            // compacted: lane j takes the j-th arc that has a gradient here
            const unsigned live = __ballot_sync(kFull, t_in);
            const int cnt = __popc(live);
            const int src = lane < cnt ? (int)__fns(live, 0, lane + 1) : lane;
            const int u_l = __shfl_sync(kFull, u_in, src);
            const int c_l = __shfl_sync(kFull, c_in, src);
            for (int j0 = 0; j0 < cnt; j0 += NG) {
                const int j = j0 + grp;
                const int u = __shfl_sync(kFull, u_l, j & 31);
                const int cu = __shfl_sync(kFull, c_l, j & 31);
                const int sj = __shfl_sync(kFull, src, j & 31);
                T acc = T(0);
                if (j < cnt) {
                    const VT *mr = reinterpret_cast<const VT *>(static_cast<const T *>(A.Mp) + (int64_t)u * A.ldp) + gl;
                    const VT *zr = reinterpret_cast<const VT *>(zb + cu * wzp) + gl;
#pragma unroll
                    for (int q = 0; q < NV; ++q) {
                        if (lim[q] > 0) {
                            const VT zq = zr[G * q];
                            const VT mq = __ldg(mr + G * q);
                            const T *zz = reinterpret_cast<const T *>(&zq);
                            const T *mm = reinterpret_cast<const T *>(&mq);
#pragma unroll
                            for (int c = 0; c < V::n; ++c)
                                if (c < lim[q]) acc = fma(zz[c], mm[c], acc);
                        }
                    }
                }
#pragma unroll
                for (int o = G >> 1; o > 0; o >>= 1) acc += __shfl_xor_sync(kFull, acc, o);
                if (gl == 0 && j < cnt) atomicAdd(A.grad + base + sj, (double)acc);  // (one term per arc)
            }
        }
        __syncwarp();
    }
}

// Per-arc weight gradient over the colour-sorted arcs (row form, p >= 2):
// the gradient of arc (v, u) is the sum over the entries e of u's compressed
// row M_p'(u, .) of M_p'(u, e) * Ybar'(v, P_e), P_e = {col u} + the e-th
// (p-1)-set of col(u)'s squeezed universe, over the sets without col(v): the
// SpMM of Alg. 4 read backwards.  v's arcs come sorted by neighbour colour,
// so each colour is one run: when a lane group's run starts, each lane reads
// the Ybar' entries its vectors pair with (the node's run map, as in the
// forward run kernel) into registers, and an arc then costs one row load per
// lane, the products and a reduction over the group.  Groups of G lanes take
// one arc each; each result goes to its arc's slot through the sort's
// permutation.  v's Ybar' row is staged in shared memory per warp, with zeros
// at ysink for the entries whose set holds col(v).
template <typename T, int G, int NV>
__global__ void __launch_bounds__(256) sddmm_sorted_kernel(const SddmmArgs A) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    using V = Vec16<T>;
    using VT = typename V::type;
    constexpr int E = V::n;
    constexpr int NG = 32 / G;
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int grp = lane / G, gl = lane % G;
    const int kc = A.kc;
    T *yb = reinterpret_cast<T *>(smem_raw) + (int64_t)wib * A.ywords;
    if (lane < E) yb[A.ysink + lane] = T(0);
    // entries of this lane's vectors inside the row (the row padding past
    // wmp is never written, and 0 times its contents need not be 0)
    int lim[NV];
#pragma unroll
    for (int q = 0; q < NV; ++q) {
        const int left = A.wmp - (gl + G * q) * E;
        lim[q] = left < 0 ? 0 : (left > E ? E : left);
    }
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t ti = (((int64_t)blockIdx.x * blockDim.x) >> 5) + wib; ti < A.ntasks; ti += nwarps) {
        const int4 task = A.tasks[ti];
        const int v = task.x;
        const int cv = A.colours[v];
        if ((unsigned)cv >= (unsigned)kc || task.z == task.w) continue;
        // the previous task's reads of yb are done
        __syncwarp();
        const T *yr = static_cast<const T *>(A.Ybar) + (int64_t)v * A.ldyb;
        for (int j = lane; j < A.ysink; j += 32) yb[j] = yr[j];
        __syncwarp();
        const uint16_t *rm = A.runmap + (int64_t)cv * kc * A.wmap + gl * E;
        T zq[NV][E];
#pragma unroll
        for (int q = 0; q < NV; ++q)
#pragma unroll
            for (int k = 0; k < E; ++k) zq[q][k] = T(0);
        int cur = -1;
        for (int64_t base = task.z; base < task.w; base += 32) {
            const int cnt_in = (int)(task.w - base < 32 ? task.w - base : 32);
            const bool in = lane < cnt_in;
            const int c_in = in ? (int)__ldg(A.sclr + base + lane) : -1;
            const bool t_in = c_in >= 0 && c_in != cv;  // (-1: a colour outside [0, kc))
            const int u_in = t_in ? __ldg(A.scol + base + lane) : 0;
            const int p_in = t_in ? __ldg(A.perm + base + lane) : 0;
            // compacted: lane j takes the j-th arc that has a gradient here
            const unsigned live = __ballot_sync(kFull, t_in);
            const int cnt = __popc(live);
            if (cnt == 0) continue;
            const int src = lane < cnt ? (int)__fns(live, 0, lane + 1) : lane;
            const int u_l = __shfl_sync(kFull, u_in, src);
            const int c_l = __shfl_sync(kFull, c_in, src);
            const int p_l = __shfl_sync(kFull, p_in, src);
            for (int j0 = 0; j0 < cnt; j0 += NG) {
                const int j = j0 + grp;
                const bool ok = j < cnt;
                const int jj = ok ? j : cnt - 1;
                const int u = __shfl_sync(kFull, u_l, jj);
                const int c = __shfl_sync(kFull, c_l, jj);
                const int pe = __shfl_sync(kFull, p_l, jj);
                if (c != cur) {
                    // the group's run changes colour: its lanes' Ybar' entries
#pragma unroll
                    for (int q = 0; q < NV; ++q) {
                        const uint16_t *mp = rm + (int64_t)c * A.wmap + G * E * q;
                        if constexpr (E == 4) {
                            const uint2 w = __ldg(reinterpret_cast<const uint2 *>(mp));
                            zq[q][0] = yb[w.x & 0xffffu];
                            zq[q][1] = yb[w.x >> 16];
                            zq[q][2] = yb[w.y & 0xffffu];
                            zq[q][3] = yb[w.y >> 16];
                        } else {
                            const uint32_t w = __ldg(reinterpret_cast<const uint32_t *>(mp));
                            zq[q][0] = yb[w & 0xffffu];
                            zq[q][1] = yb[w >> 16];
                        }
                    }
                    cur = c;
                }
                T acc = T(0);
                if (ok) {
                    const VT *mr = reinterpret_cast<const VT *>(static_cast<const T *>(A.Mp) + (int64_t)u * A.ldp) + gl;
#pragma unroll
                    for (int q = 0; q < NV; ++q) {
                        if (lim[q] > 0) {
                            const VT mq = __ldg(mr + G * q);
                            const T *mm = reinterpret_cast<const T *>(&mq);
#pragma unroll
                            for (int k = 0; k < E; ++k)
                                if (k < lim[q]) acc = fma(zq[q][k], mm[k], acc);
                        }
                    }
                }
#pragma unroll
                for (int o = G >> 1; o > 0; o >>= 1) acc += __shfl_xor_sync(kFull, acc, o);
                if (gl == 0 && ok) atomicAdd(A.grad + pe, (double)acc);  // (one term per arc)
            }
        }
    }
}

__global__ void symmetrize_kernel(const double *part, const int32_t *rev, const int32_t *arcmap, int64_t nnz,
                                  double *grad_w) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nnz; e += (int64_t)gridDim.x * blockDim.x)
        grad_w[arcmap ? (int64_t)arcmap[e] : e] = part[e] + part[rev[e]];
}

// dst[b * n + i] = src[b * n + idx[i]] for nb rows of n elements
template <typename T>
__global__ void gather_rows_kernel(const T *src, T *dst, const int32_t *idx, int64_t n, int nb) {
    const int64_t total = n * nb;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < total;
         k += (int64_t)gridDim.x * blockDim.x) {
        const int64_t b = k / n, i = k - b * n;
        dst[k] = src[b * n + idx[i]];
    }
}

// 128-bit unsigned integer to the nearest double (ties to even): the top 64
// significant bits keep a sticky bit for everything below them, so the one
// rounding of the 64-bit conversion is the correct rounding of the whole.
__global__ void finalize_kernel(const RootSum *sums, int nseg, int nb, const double *scale_hi,
                                const double *scale_lo, double *totals, double *estimates, unsigned *status) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nseg) return;
    const RootSum r = sums[s];
    double xh, xl;
    if (r.flags == 0) {
        xh = u128_to_double(r.hi, r.lo);
        // the rounding error of xh, exactly as a 128-bit difference, then to double
        unsigned long long h2 = 0, l2 = 0;
        if (xh < 0x1p64) {
            l2 = __double2ull_rz(xh);
        } else {
            const double hh = floor(xh * 0x1p-64);
            h2 = __double2ull_rz(hh);
            l2 = __double2ull_rz(xh - hh * 0x1p64);
        }
        const bool neg = (h2 > r.hi) || (h2 == r.hi && l2 > r.lo);
        unsigned long long dh, dl;
        if (!neg) {
            dl = r.lo - l2;
            dh = r.hi - h2 - (r.lo < l2 ? 1ull : 0ull);
        } else {
            dl = l2 - r.lo;
            dh = h2 - r.hi - (l2 < r.lo ? 1ull : 0ull);
        }
        xl = u128_to_double(dh, dl);
        if (neg) xl = -xl;
    } else {
        xh = r.s + r.c;
        xl = (r.s - xh) + r.c;
        if (r.flags & kFlagNonFinite) atomicOr(status, 2u);
    }
    const int pi = s / nb;
    const double sh = scale_hi[pi], sl = scale_lo[pi];
    const double p = xh * sh;
    const double e = fma(xh, sh, -p);
    totals[s] = xh;
    estimates[s] = p + (e + fma(xh, sl, xl * sh));
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

void node_shape(int vecn, int wz, int *g, int *nv) {
    const int nvec = (wz + vecn - 1) / vecn;
    *nv = 1;
    if (nvec <= 4)
        *g = 4;
    else if (nvec <= 8)
        *g = 8;
    else if (nvec <= 16)
        *g = 16;
    else {
        *g = 32;
        *nv = (nvec + 31) / 32;
        if (*nv > 4) {
            // wide: a CTA of kWideWarps warps shares the row
            *g = kWideLanes;
            *nv = (nvec + kWideWarps * 32 - 1) / (kWideWarps * 32);
            if (*nv > 4) *nv = 0;
        }
    }
}

static int blocks_per_sm_query(void *k, int threads, size_t smem) {
    if (smem > 48 * 1024) {
        // one limit per kernel variant, shared by every node that uses it: the device maximum
        int dev = 0, optin = 0;
        cudaFuncAttributes fa;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess ||
            cudaFuncGetAttributes(&fa, k) != cudaSuccess || (size_t)optin < smem + fa.sharedSizeBytes ||
            cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 optin - (int)fa.sharedSizeBytes) != cudaSuccess) {
            cudaGetLastError();
            return 0;
        }
    }
    int blocks = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, k, threads, smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return blocks;
}

// Resident blocks per SM of kernel k (0 when it cannot run with this shared
// memory), remembered per device: every request preparation asks for the same
// few launch shapes, and each driver query costs microseconds of host time.
int blocks_per_sm(void *k, int threads, size_t smem) {
    if (!k) return 0;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    static std::mutex mu;
    static std::map<std::tuple<int, void *, int, size_t>, int> known;
    const auto key = std::make_tuple(dev, k, threads, smem);
    {
        std::lock_guard<std::mutex> lock(mu);
        auto it = known.find(key);
        if (it != known.end()) return it->second;
    }
    const int blocks = blocks_per_sm_query(k, threads, smem);
    std::lock_guard<std::mutex> lock(mu);
    known[key] = blocks;
    return blocks;
}

cudaError_t launch_variant(void *k, const NodeArgs &args, int g, int threads, size_t smem, int grid_cap,
                           cudaStream_t stream) {
    if (!k) return cudaErrorInvalidValue;
    if (args.ntasks == 0) return cudaSuccess;
    // tasks per block: wide rows one per CTA, group rows 32 / g per warp, else one per warp
    const int64_t warps_per_block = g == kWideLanes ? 1 : (args.group_rows ? (threads / 32) * (32 / g) : threads / 32);
    int64_t grid = (args.ntasks + warps_per_block - 1) / warps_per_block;
    if (grid > grid_cap) grid = grid_cap;
    if (grid < 1) grid = 1;
    NodeArgs a = args;
    void *params[] = {&a};
    return cudaLaunchKernel(k, dim3((unsigned)grid), dim3((unsigned)threads), params, smem, stream);
}

int node_blocks_per_sm(Elem e, bool hist, int g, int nv, bool weighted, int threads, size_t smem, bool group) {
    return blocks_per_sm(select_kernel(e, hist, g, nv, weighted, group), threads, smem);
}

int node_blocks_per_sm_scaled(bool hist, int g, int nv, bool weighted, int threads, size_t smem, bool group) {
    return blocks_per_sm(select_kernel_scaled(hist, g, nv, weighted, group), threads, smem);
}

// The specialised epilogue a node launch can use (node_kernel's FORM).
int node_form(const NodeArgs &a, Elem e, int g, int nv) {
    if (a.group_rows && !a.hist && e != Elem::U128)
        return (a.a_leaf && !a.root && !a.defer && !a.Yout && !a.accumulate) ? 1 : 0;
    if (a.hist || a.group_rows || g != 32 || nv > 2 || e == Elem::U128) return 0;
    if (a.a_leaf && !a.root && !a.defer && !a.Yout && !a.accumulate) return 1;
    if (a.root && a.rootpair && !a.Yout && !a.defer && a.wy <= 128) return 2;
    return 0;
}

// The occupancy queries of a request configure its FORM 0 kernels; a
// specialised form chosen at launch gets its shared-memory limit raised
// here, once per kernel.
cudaError_t ensure_smem(void *k, int threads, size_t smem) {
    if (smem <= 48 * 1024) return cudaSuccess;
    static std::mutex mu;
    static std::unordered_map<void *, size_t> raised;
    std::lock_guard<std::mutex> lock(mu);
    auto it = raised.find(k);
    if (it != raised.end() && it->second >= smem) return cudaSuccess;
    if (blocks_per_sm(k, threads, smem) < 1) return cudaErrorInvalidValue;
    raised[k] = smem;
    return cudaSuccess;
}

cudaError_t launch_node(const NodeArgs &args, Elem e, int g, int nv, int threads, size_t smem, int grid_cap,
                        cudaStream_t stream) {
    const int form = node_form(args, e, g, nv);
    void *k = select_kernel(e, args.hist != 0, g, nv, args.weights != nullptr, args.group_rows != 0, form);
    if (!k) return cudaErrorInvalidValue;
    if (form != 0) {
        const cudaError_t err = ensure_smem(k, threads, smem);
        if (err != cudaSuccess) return err;
    }
    return launch_variant(k, args, g, threads, smem, grid_cap, stream);
}

cudaError_t launch_node_scaled(const NodeArgs &args, int g, int nv, int threads, size_t smem, int grid_cap,
                               cudaStream_t stream) {
    void *k = select_kernel_scaled(args.hist != 0, g, nv, args.weights != nullptr, args.group_rows != 0);
    return launch_variant(k, args, g, threads, smem, grid_cap, stream);
}

namespace {
void *select_hist_rows(Elem e, bool scaled, bool weighted) {
    if (scaled) return weighted ? reinterpret_cast<void *>(&hist_rows_kernel<float, true, true>)
                                : reinterpret_cast<void *>(&hist_rows_kernel<float, false, true>);
    if (e == Elem::U64) return weighted ? nullptr : reinterpret_cast<void *>(&hist_rows_kernel<u64, false, false>);
    if (e == Elem::U128) return weighted ? nullptr : reinterpret_cast<void *>(&hist_rows_kernel<u128, false, false>);
    if (e == Elem::F64) return weighted ? reinterpret_cast<void *>(&hist_rows_kernel<double, true, false>)
                              : reinterpret_cast<void *>(&hist_rows_kernel<double, false, false>);
    return weighted ? reinterpret_cast<void *>(&hist_rows_kernel<float, true, false>)
                    : reinterpret_cast<void *>(&hist_rows_kernel<float, false, false>);
}
}  // namespace

int hist_rows_blocks_per_sm(Elem e, bool scaled, bool weighted, int threads, size_t smem) {
    return blocks_per_sm(select_hist_rows(e, scaled, weighted), threads, smem);
}

cudaError_t launch_hist_rows(const NodeArgs &args, Elem e, bool scaled, int threads, size_t smem, int grid_cap,
                             cudaStream_t stream) {
    void *k = select_hist_rows(e, scaled, args.weights != nullptr);
    if (!k) return cudaErrorInvalidValue;
    if (args.ntasks == 0) return cudaSuccess;
    const int64_t warps = (args.ntasks + kHistRows - 1) / kHistRows;
    int64_t grid = (warps + threads / 32 - 1) / (threads / 32);
    if (grid > grid_cap) grid = grid_cap;
    if (grid < 1) grid = 1;
    NodeArgs a = args;
    void *params[] = {&a};
    return cudaLaunchKernel(k, dim3((unsigned)grid), dim3((unsigned)threads), params, smem, stream);
}

size_t ema_rows_smem(const NodeArgs &a, Elem e, bool scaled) {
    (void)scaled;
    const size_t words = (size_t)kEmaRows * (a.wy + a.Wa);
    return words * (e == Elem::F32 ? 4 : (e == Elem::U128 ? 16 : 8));
}

namespace {
void *select_ema_rows(Elem e, bool scaled) {
    if (scaled) return reinterpret_cast<void *>(&ema_rows_kernel<float, true>);
    if (e == Elem::U64) return reinterpret_cast<void *>(&ema_rows_kernel<u64, false>);
    if (e == Elem::U128) return reinterpret_cast<void *>(&ema_rows_kernel<u128, false>);
    return e == Elem::F64 ? reinterpret_cast<void *>(&ema_rows_kernel<double, false>)
                          : reinterpret_cast<void *>(&ema_rows_kernel<float, false>);
}
}  // namespace

int ema_rows_blocks_per_sm(Elem e, bool scaled, size_t smem) {
    return blocks_per_sm(select_ema_rows(e, scaled), 256, smem);
}

cudaError_t launch_ema_rows(const NodeArgs &args, Elem e, bool scaled, int sms, cudaStream_t stream) {
    const size_t smem = ema_rows_smem(args, e, scaled);
    const int per_sm = ema_rows_blocks_per_sm(e, scaled, smem);
    if (per_sm < 1) return cudaErrorInvalidValue;
    const int64_t rows = args.live_rows * args.nb;
    const int64_t blocks = std::min<int64_t>((rows + kEmaRows - 1) / kEmaRows, (int64_t)sms * per_sm);
    NodeArgs a = args;
    void *params[] = {&a};
    return cudaLaunchKernel(select_ema_rows(e, scaled), dim3((unsigned)std::max<int64_t>(blocks, 1)), dim3(256),
                            params, smem, stream);
}

cudaError_t launch_root_reduce(const void *vals, Elem ve, int64_t n, int64_t live, int nseg, double *pv,
                               const int32_t *pvmap, RootSum *partials, int chunks, RootSum *out,
                               cudaStream_t stream) {
    dim3 grid((unsigned)chunks, (unsigned)nseg);
    if (ve == Elem::U64)
        root_partial_kernel<u64><<<grid, 256, 0, stream>>>(static_cast<const u64 *>(vals), n, live, pv, pvmap, partials,
                                                             chunks);
    else if (ve == Elem::U128)
        root_partial_kernel<u128><<<grid, 256, 0, stream>>>(static_cast<const u128 *>(vals), n, live, pv, pvmap, partials,
                                                              chunks);
    else if (ve == Elem::F64)
        root_partial_kernel<double><<<grid, 256, 0, stream>>>(static_cast<const double *>(vals), n, live, pv, pvmap,
                                                                partials, chunks);
    else
        root_partial_kernel<float><<<grid, 256, 0, stream>>>(static_cast<const float *>(vals), n, live, pv, pvmap,
                                                               partials, chunks);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    root_final_kernel<<<(unsigned)nseg, 256, 0, stream>>>(partials, chunks, nseg, out);
    return cudaGetLastError();
}

cudaError_t launch_eref(const int4 *tasks, int64_t ntasks, const int32_t *scol, const int8_t *sclr,
                        const int8_t *colours, int64_t n, int64_t nnz, int nb, int kc, const int16_t *Ep,
                        int32_t *Eref, int sms, cudaStream_t stream) {
    if (ntasks == 0 || nb == 0) return cudaSuccess;
    const int64_t warps = ntasks * nb;
    int64_t grid = (warps + 7) / 8;
    const int64_t cap = (int64_t)sms * 8;
    if (grid > cap) grid = cap;
    eref_kernel<<<(unsigned)grid, 256, 0, stream>>>(tasks, ntasks, scol, sclr, colours, n, nnz, nb, kc, Ep, Eref);
    return cudaGetLastError();
}

namespace {

// The (2, 1, 1) table of a weighted graph from the colour-sorted arcs (the
// colour histogram of Sec. 4 with the weights A.val of Alg. 4): for row v and
// each colour x other than col(v), the sum of the weights of v's arcs to
// neighbours of colour x.  The arcs of a task come sorted by neighbour colour
// (invalid colours last), so each colour is one run, summed by a segmented
// scan over each batch of arcs and then batch by batch, an order that does not
// depend on scheduling.  Blocks below long_blocks take the tasks before
// small_begin, one per warp in batches of 32 arcs; the others take the tasks
// of at most kSortSmallArcs arcs from small_begin on, one per group of 8 lanes.
// Chunks of a split row add their sums into a zeroed row.  With a leaf active
// child the node's Y' row holds the same values (entry j: the j-th colour
// other than col(v)); out2, when given, receives it too.
template <typename T, int G>
__device__ __forceinline__ void weighted_hist_task(const int4 &task, bool have, int gl, T *tot,
                                                   const int8_t *__restrict__ sclr, const float *__restrict__ sw,
                                                   int64_t nnz, const int8_t *__restrict__ colours, int64_t n, int nb,
                                                   int kc, T *out, int64_t ld, T *out2, int64_t ld2) {
    const int v = task.x;
    // batches of G arcs of the longest task among the warp's groups
    const int nbat = (int)__reduce_max_sync(kFull, have ? (unsigned)((task.w - task.z + G - 1) / G) : 0u);
    for (int b = 0; b < nb; ++b) {
        const int cv = have ? (int)colours[(int64_t)b * n + v] : -1;
        const bool ok = (unsigned)cv < (unsigned)kc;
        for (int j = gl; j <= kMaxHistColours; j += G) tot[j] = T(0);
        __syncwarp();
        const int8_t *cl = sclr + (int64_t)b * nnz;
        const float *wl = sw + (int64_t)b * nnz;
        for (int kb = 0; kb < nbat; ++kb) {
            const int64_t e = task.z + (int64_t)G * kb + gl;
            const bool in = ok && e < task.w;
            const int c = in ? (int)__ldg(cl + e) : -1;
            T s = in ? T(__ldg(wl + e)) : T(0);
            // segmented inclusive scan: colours run in order, so equal
            // colours o lanes apart enclose only that colour
#pragma unroll
            for (int o = 1; o < G; o <<= 1) {
                const T y = __shfl_up_sync(kFull, s, o, G);
                const int cy = __shfl_up_sync(kFull, c, o, G);
                if (gl >= o && cy == c) s += y;
            }
            const int cn = __shfl_down_sync(kFull, c, 1, G);
            if (c >= 0 && (gl == G - 1 || cn != c)) tot[c] += s;  // one run end per colour
            __syncwarp();
        }
        if (have) {
            T *row = out + ((int64_t)v * nb + b) * ld;
            T *row2 = out2 ? out2 + ((int64_t)v * nb + b) * ld2 : nullptr;
            const int64_t width = out2 && ld2 > ld ? ld2 : ld;
            for (int j = gl; j < width; j += G) {
                const int x = j < cv ? j : j + 1;
                const T val = ok && j < kc - 1 ? tot[x] : T(0);
                if (task.y < 0) {
                    if (j < ld) row[j] = val;
                    if (row2 && j < ld2) row2[j] = val;
                } else if (val != T(0)) {
                    if (j < ld) atomicAdd(row + j, val);
                    if (row2 && j < ld2) atomicAdd(row2 + j, val);
                }
            }
        }
        __syncwarp();
    }
}

template <typename T>
__global__ void __launch_bounds__(256) weighted_hist_kernel(const int4 *__restrict__ tasks, int64_t ntasks,
                                                            int64_t small_begin, int64_t long_blocks,
                                                            const int8_t *__restrict__ sclr,
                                                            const float *__restrict__ sw, int64_t nnz,
                                                            const int8_t *__restrict__ colours, int64_t n, int nb,
                                                            int kc, T *out, int64_t ld, T *out2, int64_t ld2) {
    __shared__ T tot_s[8][4][kMaxHistColours + 1];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    if ((int64_t)blockIdx.x < long_blocks) {
        const int64_t nwarps = long_blocks * 8;
        for (int64_t t = (int64_t)blockIdx.x * 8 + wib; t < small_begin; t += nwarps)
            weighted_hist_task<T, 32>(tasks[t], true, lane, tot_s[wib][0], sclr, sw, nnz, colours, n, nb, kc, out, ld,
                                      out2, ld2);
        return;
    }
    constexpr int G = 8;
    const int grp = lane / G;
    const int64_t nwarps = ((int64_t)gridDim.x - long_blocks) * 8;
    const int64_t rounds = (ntasks - small_begin + 32 / G - 1) / (32 / G);
    for (int64_t rd = ((int64_t)blockIdx.x - long_blocks) * 8 + wib; rd < rounds; rd += nwarps) {
        const int64_t t = small_begin + rd * (32 / G) + grp;
        const bool have = t < ntasks;
        const int4 task = have ? tasks[t] : make_int4(0, -1, 0, 0);
        weighted_hist_task<T, G>(task, have, lane % G, tot_s[wib][grp], sclr, sw, nnz, colours, n, nb, kc, out, ld,
                                 out2, ld2);
    }
}

}  // namespace

cudaError_t launch_weighted_hist(const int4 *tasks, int64_t ntasks, int64_t small_begin, const int8_t *sclr,
                                 const float *sw, int64_t nnz, const int8_t *colours, int64_t n, int nb, int kc,
                                 void *out, int64_t ld, void *out2, int64_t ld2, Elem e, int sms,
                                 cudaStream_t stream) {
    if (ntasks <= 0) return cudaSuccess;
    if (kc > kMaxHistColours || !sw) return cudaErrorInvalidValue;
    small_begin = small_begin < 0 ? 0 : (small_begin > ntasks ? ntasks : small_begin);
    // one wave of 8 blocks per SM, split between the two kinds of task
    const int64_t cap = (int64_t)sms * (small_begin > 0 && small_begin < ntasks ? 4 : 8);
    int64_t long_blocks = (small_begin + 7) / 8;
    if (long_blocks > cap) long_blocks = cap;
    int64_t small_blocks = ((ntasks - small_begin + 3) / 4 + 7) / 8;
    if (small_blocks > cap) small_blocks = cap;
    const unsigned grid = (unsigned)(long_blocks + small_blocks);
    if (e == Elem::F64)
        weighted_hist_kernel<double><<<grid, 256, 0, stream>>>(tasks, ntasks, small_begin, long_blocks, sclr, sw, nnz,
                                                               colours, n, nb, kc, static_cast<double *>(out), ld,
                                                               static_cast<double *>(out2), ld2);
    else if (e == Elem::F32)
        weighted_hist_kernel<float><<<grid, 256, 0, stream>>>(tasks, ntasks, small_begin, long_blocks, sclr, sw, nnz,
                                                              colours, n, nb, kc, static_cast<float *>(out), ld,
                                                              static_cast<float *>(out2), ld2);
    else
        return cudaErrorInvalidValue;
    return cudaGetLastError();
}

cudaError_t launch_colour_sort(const int4 *tasks, int64_t ntasks, int64_t small_begin, const int32_t *col_idx,
                               const float *weights, int64_t n, int64_t nnz, const int8_t *colours, int nb, int kc,
                               int32_t *scol, int8_t *sclr, float *sw, const SortHist &hist, int sms,
                               cudaStream_t stream) {
    if (small_begin > 0) {
        // one wave of resident blocks (the staging buffers limit residency)
        const bool with_hist = hist.out || hist.hcount;
        // (both variants use the same staging buffers: one residency figure)
        static const int per_sm = std::max(1, blocks_per_sm(reinterpret_cast<void *>(&colour_sort_kernel<true>), 256, 0));
        int64_t blocks = (small_begin + 7) / 8;
        if (blocks > (int64_t)sms * per_sm) blocks = (int64_t)sms * per_sm;
        if (with_hist)
            colour_sort_kernel<true><<<(unsigned)blocks, 256, 0, stream>>>(tasks, small_begin, col_idx, weights, n, nnz,
                                                                           colours, nb, kc, scol, sclr, sw, hist);
        else
            colour_sort_kernel<false><<<(unsigned)blocks, 256, 0, stream>>>(tasks, small_begin, col_idx, weights, n, nnz,
                                                                            colours, nb, kc, scol, sclr, sw, hist);
    }
    const int64_t rest = ntasks - small_begin;
    if (rest > 0) {
        constexpr int G = kSortSmallArcs;
        int64_t blocks = ((rest + 32 / G - 1) / (32 / G) + 7) / 8;
        if (blocks > (int64_t)sms * 16) blocks = (int64_t)sms * 16;
        colour_sort_small_kernel<G><<<(unsigned)blocks, 256, 0, stream>>>(
            tasks + small_begin, rest, col_idx, weights, n, nnz, colours, nb, kc, scol, sclr, sw, hist);
    }
    return cudaGetLastError();
}

cudaError_t launch_finalize(const RootSum *sums, int nseg, int nb, const double *scale_hi, const double *scale_lo,
                            double *totals, double *estimates, unsigned *status, cudaStream_t stream) {
    finalize_kernel<<<(nseg + 127) / 128, 128, 0, stream>>>(sums, nseg, nb, scale_hi, scale_lo, totals, estimates,
                                                            status);
    return cudaGetLastError();
}

cudaError_t launch_bwd_ema(const BwdEmaArgs &args, bool fp64, int sms, cudaStream_t stream) {
    const size_t smem = (size_t)8 * (args.ws + args.wa + args.wy) * (fp64 ? 8 : 4);
    void *k = fp64 ? reinterpret_cast<void *>(&bwd_ema_kernel<double>)
                   : reinterpret_cast<void *>(&bwd_ema_kernel<float>);
    // (raises the kernel's shared-memory limit past 48 KB when the rows need it)
    const int per_sm = blocks_per_sm(k, 256, smem);
    if (per_sm < 1) return cudaErrorInvalidValue;
    const int64_t blocks = std::min<int64_t>((args.n + 7) / 8, (int64_t)sms * per_sm);
    BwdEmaArgs a = args;
    void *params[] = {&a};
    return cudaLaunchKernel(k, dim3((unsigned)std::max<int64_t>(blocks, 1)), dim3(256), params, smem, stream);
}

namespace {
template <typename T>
void *pick_sddmm_rows(int g, int nv) {
    if (g == 4) return reinterpret_cast<void *>(&sddmm_rows_kernel<T, 4, 1>);
    if (g == 8) return reinterpret_cast<void *>(&sddmm_rows_kernel<T, 8, 1>);
    if (g == 16) return reinterpret_cast<void *>(&sddmm_rows_kernel<T, 16, 1>);
    if (g != 32) return nullptr;
    switch (nv) {
        case 1: return reinterpret_cast<void *>(&sddmm_rows_kernel<T, 32, 1>);
        case 2: return reinterpret_cast<void *>(&sddmm_rows_kernel<T, 32, 2>);
        case 3: return reinterpret_cast<void *>(&sddmm_rows_kernel<T, 32, 3>);
        case 4: return reinterpret_cast<void *>(&sddmm_rows_kernel<T, 32, 4>);
        default: return nullptr;
    }
}
template <typename T>
void *pick_sddmm_sorted(int g, int nv) {
    if (nv == 1) {
        if (g == 4) return reinterpret_cast<void *>(&sddmm_sorted_kernel<T, 4, 1>);
        if (g == 8) return reinterpret_cast<void *>(&sddmm_sorted_kernel<T, 8, 1>);
        if (g == 16) return reinterpret_cast<void *>(&sddmm_sorted_kernel<T, 16, 1>);
        if (g == 32) return reinterpret_cast<void *>(&sddmm_sorted_kernel<T, 32, 1>);
    }
    if (nv == 2 && g == 32) return reinterpret_cast<void *>(&sddmm_sorted_kernel<T, 32, 2>);
    return nullptr;
}
}  // namespace

bool sddmm_sorted_available(bool fp64, int lanes, int vecs) {
    return (fp64 ? pick_sddmm_sorted<double>(lanes, vecs) : pick_sddmm_sorted<float>(lanes, vecs)) != nullptr;
}

cudaError_t launch_sddmm(const SddmmArgs &args, bool fp64, int sms, cudaStream_t stream) {
    if (!args.hist && args.tasks && args.lanes > 0 && args.scol) {
        // sorted form
        void *k = fp64 ? pick_sddmm_sorted<double>(args.lanes, args.vecs)
                       : pick_sddmm_sorted<float>(args.lanes, args.vecs);
        if (!k || !args.runmap || !args.perm) return cudaErrorInvalidValue;
        if (args.ntasks == 0) return cudaSuccess;
        const size_t smem = (size_t)8 * args.ywords * (fp64 ? 8 : 4);
        const int per_sm = blocks_per_sm(k, 256, smem);
        if (per_sm < 1) return cudaErrorInvalidValue;
        const int64_t blocks = std::min<int64_t>((args.ntasks + 7) / 8, (int64_t)sms * per_sm);
        SddmmArgs a = args;
        void *params[] = {&a};
        return cudaLaunchKernel(k, dim3((unsigned)std::max<int64_t>(blocks, 1)), dim3(256), params, smem, stream);
    }
    if (!args.hist && args.tasks && args.lanes > 0) {
        // row-oriented form
        void *k = fp64 ? pick_sddmm_rows<double>(args.lanes, args.vecs) : pick_sddmm_rows<float>(args.lanes, args.vecs);
        const size_t smem = (size_t)8 * args.kc * args.wz_pad * (fp64 ? 8 : 4);
        if (!k) return cudaErrorInvalidValue;
        if (args.ntasks == 0) return cudaSuccess;
        // (raises the kernel's shared-memory limit when it needs more than 48 KB)
        const int per_sm = blocks_per_sm(k, 256, smem);
        if (per_sm < 1) return cudaErrorInvalidValue;
        const int64_t blocks = std::min<int64_t>((args.ntasks + 7) / 8, (int64_t)sms * std::max(per_sm, 1));
        SddmmArgs a = args;
        void *params[] = {&a};
        return cudaLaunchKernel(k, dim3((unsigned)std::max<int64_t>(blocks, 1)), dim3(256), params, smem, stream);
    }
    const size_t smem = (size_t)8 * ((args.wmp + 3) / 4 * 4) * (fp64 ? 8 : 4);
    if (smem > 48 * 1024) return cudaErrorInvalidValue;
    const int64_t units = args.tasks ? args.ntasks : args.n;
    const int64_t blocks = std::min<int64_t>((units + 7) / 8, (int64_t)sms * 8);
    if (fp64)
        sddmm_kernel<double><<<(unsigned)std::max<int64_t>(blocks, 1), 256, smem, stream>>>(args);
    else
        sddmm_kernel<float><<<(unsigned)std::max<int64_t>(blocks, 1), 256, smem, stream>>>(args);
    return cudaGetLastError();
}

template <typename T>
cudaError_t gather_rows(const T *src, T *dst, const int32_t *idx, int64_t n, int nb, cudaStream_t stream) {
    if (n == 0 || nb == 0) return cudaSuccess;
    int64_t blocks = (n * nb + 255) / 256;
    if (blocks > 8192) blocks = 8192;
    gather_rows_kernel<T><<<(unsigned)blocks, 256, 0, stream>>>(src, dst, idx, n, nb);
    return cudaGetLastError();
}

cudaError_t launch_gather_i8(const int8_t *src, int8_t *dst, const int32_t *idx, int64_t n, int nb,
                             cudaStream_t stream) {
    return gather_rows<int8_t>(src, dst, idx, n, nb, stream);
}
cudaError_t launch_gather_f32(const float *src, float *dst, const int32_t *idx, int64_t n, cudaStream_t stream) {
    return gather_rows<float>(src, dst, idx, n, 1, stream);
}
cudaError_t launch_gather_f64(const double *src, double *dst, const int32_t *idx, int64_t n, cudaStream_t stream) {
    return gather_rows<double>(src, dst, idx, n, 1, stream);
}

cudaError_t launch_symmetrize(const double *part, const int32_t *rev, const int32_t *arcmap, int64_t nnz,
                              double *grad_w, cudaStream_t stream) {
    if (nnz == 0) return cudaSuccess;
    const int64_t blocks = std::min<int64_t>((nnz + 255) / 256, 4096);
    symmetrize_kernel<<<(unsigned)blocks, 256, 0, stream>>>(part, rev, arcmap, nnz, grad_w);
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
