// Run-scatter node kernel: one launch per DP node (Alg. 5) for the gathering
// nodes of plain FP32 / FP64 tables.
//
// A warp owns one work-list task (a row v, or a chunk of a long row) and
// computes, for the node s = (T_s, T_a, T_p),
//   Y'(v, P)   = sum over arcs (v, u) of w_vu * M_p'(u, P - {col(u)})   (Alg. 4 / 6)
//   M_s'(v, S) = sum over splits of M_a'(v, A) * Y'(v, S - A)           (Eq. 1)
// in the colour-compressed layout (row v keeps only the sets holding
// col(v)).  The arcs of a task come sorted by neighbour colour, so each colour
// d is one run (per lane group), summed in registers; when the run ends, its
// sum Z(d, .) goes straight to where the eMA needs it, through the node's run
// map for the pair (col(v), d):
//   FORM 0 / 1: Y'(P) += Z(d, P - {d}) for the p-sets P without col(v)
//               (Y' in shared memory; FORM 1, a single-vertex active child,
//               stores Y' as the output row, FORM 0 runs the eMA epilogue);
//   FORM 2:     a root with one output set: the row sum gains
//               Z(d, Q) * M_a'(v, S' - Q - {d}) for every (p-1)-set Q
//               without col(v) (the active row in shared memory).
// Entries of Z(d) whose set holds col(v) map to a sink (a Y' slot nothing
// reads, or a zero of the active row), so the scatter has no branches.  No
// per-colour accumulators are kept, so rows with few colours pay only for the
// colours they have.
//
// Lanes form groups of G that cover one neighbour row (G * NV 16-byte
// vectors), so a warp instruction gathers 32 / G arcs (group g takes every
// (32/G)-th arc of the task, so every group walks the same colour runs).
// The gather loop is kept short because these launches are bound by issue
// slots: each
// batch of 32 sorted arcs is compacted (through shared memory) to the arcs
// that add something, each as one word (u * vectors per vertex) << 4 |
// colour (below 2^28 vectors: the launcher checks), so an arc costs one
// shuffle, one address, one 16-byte load and the adds; lanes past the row's
// last vector load that vector again (no predicate), and a step that stays
// in every group's current run skips the per-arc colour test.  Groups
// narrower than the warp end their runs at different times, so each scatters
// into its own copy of Y'; the copies are summed once the task's arcs are
// done.
#include <cuda_runtime.h>

#include <cstdint>

#include "device_common.cuh"
#include "kernels.cuh"

namespace sg2v {

namespace {

#ifndef SG2V_RUN_MINB_F32
#define SG2V_RUN_MINB_F32 5
#endif
#ifndef SG2V_RUN_U_F32
#define SG2V_RUN_U_F32 4
#endif
// warp-wide groups scatter with plain read-modify-writes (1) or atomics (0)
#ifndef SG2V_RUN_RMW32
#define SG2V_RUN_RMW32 1
#endif
#ifndef SG2V_RUN_BLOCKS
#define SG2V_RUN_BLOCKS 1
#endif

// Resident blocks per SM requested from the compiler (the register cap);
// tuned on B300 (occupancy matters more than a few spills).
template <typename T, int NV>
struct RunMinBlocks {
    static constexpr int value = sizeof(T) == 4 ? SG2V_RUN_MINB_F32 : (NV == 1 ? 3 : 2);
};

// L2 cache policies (createpolicy): evict-first for data used once per
// launch, evict-normal otherwise.
__device__ __forceinline__ uint64_t l2_policy(bool evict_first) {
    uint64_t p;
    if (evict_first)
        asm("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    else
        asm("createpolicy.fractional.L2::evict_normal.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ int ld_hint_s8(const int8_t *p, uint64_t pol) {
    int v;
    asm("ld.global.nc.L2::cache_hint.s8 %0, [%1], %2;" : "=r"(v) : "l"(p), "l"(pol));
    return v;
}
__device__ __forceinline__ int ld_hint_s32(const int32_t *p, uint64_t pol) {
    int v;
    asm("ld.global.nc.L2::cache_hint.b32 %0, [%1], %2;" : "=r"(v) : "l"(p), "l"(pol));
    return v;
}
template <typename VT>
__device__ __forceinline__ void st_hint_v16(VT *p, const VT &x, uint64_t pol) {
    static_assert(sizeof(VT) == 16, "16-byte vectors");
    const uint4 w = *reinterpret_cast<const uint4 *>(&x);
    asm volatile("st.global.L2::cache_hint.v4.b32 [%0], {%1, %2, %3, %4}, %5;" ::"l"(p), "r"(w.x), "r"(w.y), "r"(w.z),
                 "r"(w.w), "l"(pol)
                 : "memory");
}

template <typename T, int G, int NV, bool WEIGHTED, int FORM>
__global__ void __launch_bounds__(kNodeThreads, RunMinBlocks<T, NV>::value) node_run_kernel(const NodeArgs A) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    using V = Vec16<T>;
    using VT = typename V::type;
    constexpr int E = V::n;    // entries per 16-byte vector
    constexpr int NG = 32 / G; // arcs per warp instruction
    constexpr int U = (NV == 1 && sizeof(T) == 4 && G == 32) ? SG2V_RUN_U_F32 : 4;  // arcs in flight per group and step
    // FP64 adds are scarce on this part: slots past a batch's live arcs skip
    // their load and adds; FP32 slots read the zero row instead
    constexpr bool SKIP_ZERO = sizeof(T) >= 8;
    // warp-wide groups scatter with plain read-modify-writes (or atomics when
    // SG2V_RUN_RMW32 = 0); narrower groups each own a copy of Y' (no group
    // races another), folded once the task's arcs are done
    constexpr bool RMW = G < 32 || SG2V_RUN_RMW32;
    static_assert(32 % (NG * U) == 0, "a step's arcs must stay inside one batch of 32");
    static_assert(G != 32 || U % 4 == 0, "warp-wide groups read a step's packed arcs four at a time");
    // narrower groups take a block of U consecutive slots per step (group g:
    // slots g U .. g U + U - 1) and read them with one 16-byte shared load;
    // SG2V_RUN_BLOCKS=0 deals the slots round-robin through shuffles
    constexpr bool SLOTS = G == 32 || (SG2V_RUN_BLOCKS && U == 4);
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const int grp = lane / G, gl = lane % G;
    // per warp: Y' with its sink (FORM 0 / 1), the active row with its zero
    // (a >= 2 or FORM 2), and the batch's compacted arcs
    const int yreg = NG * A.ywords;  // Y' copies of the warp's groups
    T *ybuf = reinterpret_cast<T *>(smem_raw) + (int64_t)wib * (yreg + A.mwords);
    T *mbuf = ybuf + yreg;
    T *ygrp = ybuf + grp * A.ywords;  // this group's copy
    const unsigned gmask = (G == 32 ? kFull : ((1u << G) - 1u)) << (grp * G);
    unsigned *cbuf = reinterpret_cast<unsigned *>(reinterpret_cast<unsigned char *>(smem_raw) +
                                                  (size_t)(blockDim.x >> 5) * (NG * A.ywords + A.mwords) * sizeof(T) +
                                                  (size_t)wib * kRunCompactBytes);
    float *wbuf = reinterpret_cast<float *>(cbuf + 32);
    // the warp's next task descriptor, copied in while the current task runs
    // (kept out of registers: they are the kernel's scarce resource)
    int4 *nslot = reinterpret_cast<int4 *>(cbuf + 64);
    const int kc = A.kc;
    const int mchunks = (A.a_leaf || A.defer) ? 0 : (A.Wa * (int)sizeof(T) + 15) / 16;
    const int nvec = (A.Wz + E - 1) / E;
    const uint32_t sink = (uint32_t)(A.ywords - E);  // the run map's Y' sink (forms 0 and 1)
    // the vector each lane loads (lanes past the row's end repeat the last
    // one: same line, no extra traffic) and which of its entries are real
    int lv_[NV];
    unsigned emask = 0;
#pragma unroll
    for (int q = 0; q < NV; ++q) {
        lv_[q] = min(gl + G * q, nvec - 1);
#pragma unroll
        for (int k = 0; k < E; ++k)
            if ((gl + G * q) * E + k < A.Wz) emask |= 1u << (q * E + k);
    }
    if (FORM == 2) {
        // the active row's zero (the sink of the dot products); a single-vertex
        // active child is the one-entry row {1}
        if (lane < E) mbuf[A.mzero + lane] = T(0);
        if (A.a_leaf && lane == 0) mbuf[0] = T(1);
    }
    // packed arcs carry the gathered row's first vector, u * uvec (the launcher
    // keeps (n + 1) * uvec below 2^28), so an arc's address is one multiply-add
    const unsigned zero_word = ((unsigned)A.n * A.uvec) << 4;      // the zero row
    const uint64_t pol_once = l2_policy(A.l2_stream != 0);
    // (a work list has fewer than 2^32 tasks: one per row plus the chunks)
    const unsigned nwarps = (gridDim.x * blockDim.x) >> 5;
    const unsigned ntasks = (unsigned)A.ntasks;
    unsigned ti = ((blockIdx.x * blockDim.x) >> 5) + wib;
    int4 task = ti < ntasks ? A.tasks[ti] : make_int4(0, -1, 0, 0);
    unsigned ovf = 0;
    for (; ti < ntasks; ti += nwarps) {
        const bool more = ti + nwarps < ntasks;
        if (more && lane == 0) {
            const unsigned dst = (unsigned)__cvta_generic_to_shared(nslot);
            asm volatile("cp.async.ca.shared.global [%0], [%1], 16;\n" ::"r"(dst), "l"(A.tasks + ti + nwarps)
                         : "memory");
        }
        asm volatile("cp.async.commit_group;\n" ::: "memory");
        const int v = task.x;
        const int slot = task.y;
        const int64_t e0 = task.z, e1 = task.w;
        for (int b = 0; b < A.nb; ++b) {
            const int64_t rowb = (int64_t)v * A.nb + b;
            const int cv = A.colours[(int64_t)b * A.n + v];
            const bool cok = (unsigned)cv < (unsigned)kc;
            if (slot < 0 && (e0 == e1 || !cok)) {
                // no arcs (or no valid colour): every output of the row is zero
                if (A.defer) {
                    T *yo = static_cast<T *>(A.Yout) + rowb * A.ldy;
                    for (int j = lane; j < A.wy; j += 32) yo[j] = T(0);
                } else if constexpr (FORM == 2) {
                    if (lane == 0) static_cast<T *>(A.root_out)[(int64_t)b * A.n + v] = T(0);
                } else if constexpr (FORM == 1) {
                    // (an accumulated output keeps its row: nothing to add)
                    VT *out = reinterpret_cast<VT *>(static_cast<T *>(A.Ms) + rowb * A.ldt);
                    if (!A.accumulate)
                        for (int j = lane; j < (A.ywords - E) / E; j += 32) out[j] = V::zero();
                } else {
                    epilogue<T>(A, v, b, false, ybuf, mbuf, lane, ovf);
                }
                __syncwarp();
                continue;
            }
            if (mchunks && cok) {
                // the active row, needed by the eMA (and by FORM 2's runs)
                const char *src = static_cast<const char *>(A.Ma) + rowb * A.lda * sizeof(T);
                for (int c = lane; c < mchunks; c += 32) {
                    const unsigned dst = (unsigned)__cvta_generic_to_shared(reinterpret_cast<char *>(mbuf) + 16 * c);
                    asm volatile("cp.async.cg.shared.global.L2::cache_hint [%0], [%1], 16, %2;\n" ::"r"(dst),
                                 "l"(src + 16 * c), "l"(pol_once)
                                 : "memory");
                }
                asm volatile("cp.async.commit_group;\n" ::: "memory");
            }
            if (FORM != 2)
                for (int j = lane; j < yreg; j += 32) ybuf[j] = T(0);
            bool mready = mchunks == 0 || !cok;
            T acc = T(0);  // FORM 2: this lane's part of the row sum
            // lane vectors as 32-bit offsets from the table (fewer live registers)
            unsigned lvo[NV];
#pragma unroll
            for (int q = 0; q < NV; ++q) lvo[q] = (unsigned)(b * A.ldp / E) + (unsigned)lv_[q];
            // the task's sorted arcs (a task holds at most a chunk of arcs:
            // 32-bit offsets from its first arc)
            const int64_t aoff = (int64_t)b * A.nnz + e0;
            const int len = (int)(e1 - e0);
            const unsigned rmo = (unsigned)((cok ? cv : 0) * kc * A.wmap + gl * E);
            VT run[NV];
#pragma unroll
            for (int q = 0; q < NV; ++q) run[q] = V::zero();
            int cur = -1;
            // the end of a colour run of this lane's group (called by the
            // group's lanes only; warp-wide groups call it uniformly)
            auto flush = [&](int c) {
                const uint16_t *mp = A.runmap + (rmo + (unsigned)(c * A.wmap));
#pragma unroll
                for (int q = 0; q < NV; ++q) {
                    uint32_t ix[E];
                    if constexpr (E == 4) {
                        const uint2 w = __ldg(reinterpret_cast<const uint2 *>(mp + G * E * q));
                        ix[0] = w.x & 0xffffu;
                        ix[1] = w.x >> 16;
                        ix[2] = w.y & 0xffffu;
                        ix[3] = w.y >> 16;
                    } else {
                        const uint32_t w = __ldg(reinterpret_cast<const uint32_t *>(mp + G * E * q));
                        ix[0] = w & 0xffffu;
                        ix[1] = w >> 16;
                    }
                    const T *rv = reinterpret_cast<const T *>(&run[q]);
#pragma unroll
                    for (int k = 0; k < E; ++k) {
                        if constexpr (FORM == 2) {
                            // entries past the row (padding) may hold anything
                            const T x = (emask >> (q * E + k) & 1u) ? rv[k] : T(0);
                            acc = fma(x, mbuf[ix[k]], acc);
                        } else if constexpr (RMW) {
                            ygrp[ix[k]] += rv[k];
                        } else {
                            // one shared-memory reduction per entry; the sink's
                            // entries are skipped (their adds would serialise)
                            if (ix[k] != sink) atomicAdd(ybuf + ix[k], rv[k]);
                        }
                    }
                    run[q] = V::zero();
                }
                // the next run may add to the same entries of Y'
                if (FORM != 2 && RMW) __syncwarp(gmask);
            };
            for (int base = 0; base < len; base += 32) {
                const int cnt_in = len - base < 32 ? len - base : 32;
                const bool in = lane < cnt_in;
                const int c_in = in ? ld_hint_s8(A.sclr + aoff + base + lane, pol_once) : -1;
                const int u_in = in ? ld_hint_s32(A.scol + aoff + base + lane, pol_once) : 0;
                const bool t_in = cok && c_in >= 0 && c_in != cv && (!A.half_arcs || u_in < v);
                // compact the batch to the arcs that add something (order kept,
                // so colour runs stay contiguous) through the warp's slots
                const unsigned live = __ballot_sync(kFull, t_in);
                const int cnt = __popc(live);
                if (cnt == 0) continue;
                if (t_in) {
                    const int r = __popc(live & ((1u << lane) - 1u));
                    cbuf[r] = (((unsigned)u_in * A.uvec) << 4) | (unsigned)c_in;
                    if (WEIGHTED) wbuf[r] = __ldg(A.sw + aoff + base + lane);
                }
                __syncwarp();
                // slots past the live arcs read the zero row into the batch's
                // last run, so a run that continues in the next batch is not cut
                unsigned pk = 0;
                T w_l = T(1);
                if constexpr (SLOTS) {
                    // the groups read the packed arcs four at a time from
                    // the slots (one broadcast load per step instead of a
                    // shuffle per arc): the padding slots are filled here
                    if (lane >= cnt) {
                        cbuf[lane] = zero_word | (cbuf[cnt - 1] & 15u);
                        if (WEIGHTED) wbuf[lane] = 0.f;
                    }
                } else {
                    const unsigned wl = cbuf[lane < cnt ? lane : cnt - 1];
                    pk = lane < cnt ? wl : (zero_word | (wl & 15u));
                    if (WEIGHTED) w_l = lane < cnt ? T(wbuf[lane]) : T(0);
                }
                __syncwarp();
                if (FORM == 2 && !mready) {
                    // the active row is read from the first run end on
                    asm volatile("cp.async.wait_all;\n" ::: "memory");
                    __syncwarp();
                    mready = true;
                }
                for (int j0 = 0; j0 < cnt; j0 += NG * U) {
                    VT x[U][NV];
                    T w[U];
                    int cr[U];
                    uint4 pw4[SLOTS ? U / 4 : 1];
                    float4 w4[SLOTS ? U / 4 : 1];
                    // this group's first slot of the step
                    const int g0s = j0 + (G == 32 ? 0 : grp * U);
                    if constexpr (SLOTS) {
#pragma unroll
                        for (int h = 0; h < U / 4; ++h) {
                            pw4[h] = *reinterpret_cast<const uint4 *>(cbuf + g0s + 4 * h);
                            if (WEIGHTED) w4[h] = *reinterpret_cast<const float4 *>(wbuf + g0s + 4 * h);
                        }
                    }
#pragma unroll
                    for (int r = 0; r < U; ++r) {
                        const int j = SLOTS ? g0s + r : j0 + r * NG + grp;
                        unsigned pw;
                        if constexpr (SLOTS) {
                            const uint4 &p4 = pw4[r / 4];
                            const int k4 = r % 4;
                            pw = k4 == 0 ? p4.x : (k4 == 1 ? p4.y : (k4 == 2 ? p4.z : p4.w));
                            if (WEIGHTED) {
                                const float4 &q4 = w4[r / 4];
                                w[r] = T(k4 == 0 ? q4.x : (k4 == 1 ? q4.y : (k4 == 2 ? q4.z : q4.w)));
                            } else {
                                w[r] = T(1);
                            }
                        } else {
                            pw = __shfl_sync(kFull, pk, j);
                            w[r] = WEIGHTED ? __shfl_sync(kFull, w_l, j) : T(1);
                        }
                        const unsigned uo = pw >> 4;  // the row's first vector
                        cr[r] = (int)(pw & 15u);
#pragma unroll
                        for (int q = 0; q < NV; ++q)
                            x[r][q] = (!SKIP_ZERO || j < cnt)
                                          ? ldg_row(reinterpret_cast<const VT *>(A.Mp) + (uo + lvo[q]))
                                          : V::zero();
                    }
                    const bool same = G == 32 ? cr[U - 1] == cur : __all_sync(kFull, cr[U - 1] == cur);
                    if (same) {
                        // the whole step continues every group's current run
#pragma unroll
                        for (int r = 0; r < U; ++r) {
                            if (SKIP_ZERO && (SLOTS ? g0s + r : j0 + r * NG + grp) >= cnt) continue;
#pragma unroll
                            for (int q = 0; q < NV; ++q) {
                                if (WEIGHTED)
                                    V::fma(run[q], w[r], x[r][q]);
                                else
                                    V::add(run[q], x[r][q]);
                            }
                        }
                    } else {
#pragma unroll
                        for (int r = 0; r < U; ++r) {
                            if (SKIP_ZERO && (SLOTS ? g0s + r : j0 + r * NG + grp) >= cnt) continue;
                            if (cr[r] != cur) {
                                if (cur >= 0) flush(cur);
                                cur = cr[r];
                            }
#pragma unroll
                            for (int q = 0; q < NV; ++q) {
                                if (WEIGHTED)
                                    V::fma(run[q], w[r], x[r][q]);
                                else
                                    V::add(run[q], x[r][q]);
                            }
                        }
                    }
                }
                // every lane has read the slots before the next batch refills them
                if constexpr (SLOTS) __syncwarp();
            }
            if (cur >= 0) flush(cur);
            if (FORM == 2 && !mready) asm volatile("cp.async.wait_all;\n" ::: "memory");
            __syncwarp();
            if constexpr (NG > 1 && FORM != 2) {
                // fold the groups' copies of Y' into the first
                for (int j = lane; j < A.ywords; j += 32) {
                    T y = ybuf[j];
#pragma unroll
                    for (int g2 = 1; g2 < NG; ++g2) y += ybuf[g2 * A.ywords + j];
                    ybuf[j] = y;
                }
                __syncwarp();
            }
            if constexpr (FORM == 2) {
                T s = warp_sum(acc);
                if (slot >= 0) {
                    // one chunk of a split row: its part of the row sum goes to
                    // the scratch row; the last chunk to arrive writes the sum
                    T *sc = static_cast<T *>(A.scratch) + ((int64_t)slot * A.nb + b) * A.scratch_ld;
                    int last = 0;
                    if (lane == 0) {
                        atomicAdd(sc, s);
                        __threadfence();
                        const unsigned done = atomicAdd(A.counters + (int64_t)slot * A.nb + b, 1u);
                        last = (done + 1u == (unsigned)__ldg(A.heavy_chunks + slot));
                        if (last) {
                            __threadfence();
                            s = __ldcg(sc);
                        }
                    }
                    last = __shfl_sync(kFull, last, 0);
                    if (!last) {
                        __syncwarp();
                        continue;
                    }
                }
                if (lane == 0)
                    static_cast<T *>(A.root_out)[(int64_t)b * A.n + v] = cok ? (A.half_arcs ? T(2) * s : s) : T(0);
                __syncwarp();
                continue;
            }
            if (slot >= 0) {
                // one chunk of a split row: fold Y' into the scratch row; the
                // last chunk to arrive finishes the row
                T *sc = static_cast<T *>(A.scratch) + ((int64_t)slot * A.nb + b) * A.scratch_ld;
                if (cok)
                    for (int j = lane; j < A.wy; j += 32) atomicAdd(sc + j, ybuf[j]);
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
                for (int j = lane; j < A.wy; j += 32) ybuf[j] = __ldcg(sc + j);
                __syncwarp();
            }
            if constexpr (FORM == 1) {
                // M_s' = Y' (the row's padding gets Y's zeros)
                VT *out = reinterpret_cast<VT *>(static_cast<T *>(A.Ms) + rowb * A.ldt);
                const VT *yv = reinterpret_cast<const VT *>(ybuf);
                // (the Y' vectors: the output row's width rounded to whole vectors)
                const int nout = (A.ywords - E) / E;
                if (A.accumulate) {
                    // the backward's transposed SpMM adds to the gradient row
                    if (cok)
                        for (int j = lane; j < nout; j += 32) {
                            VT o = out[j];
                            V::add(o, yv[j]);
                            out[j] = o;
                        }
                } else {
                    for (int j = lane; j < nout; j += 32) st_hint_v16(out + j, cok ? yv[j] : V::zero(), pol_once);
                }
                __syncwarp();
                continue;
            }
            if (mchunks && cok) asm volatile("cp.async.wait_all;\n" ::: "memory");
            __syncwarp();
            if (A.defer) {
                // the eMA runs in its own launch over blocks of rows
                T *yo = static_cast<T *>(A.Yout) + rowb * A.ldy;
                for (int j = lane; j < A.wy; j += 32) yo[j] = cok ? ybuf[j] : T(0);
                __syncwarp();
                continue;
            }
            epilogue<T>(A, v, b, cok, ybuf, mbuf, lane, ovf);
            __syncwarp();
        }
        asm volatile("cp.async.wait_all;\n" ::: "memory");
        __syncwarp();
        if (more) task = *nslot;
        // every lane has read the slot before the next copy overwrites it
        __syncwarp();
    }
}

template <typename T, int G, int NV, bool W>
void *pick_form(int form) {
    if (form == 1) return reinterpret_cast<void *>(&node_run_kernel<T, G, NV, W, 1>);
    if (form == 2) return reinterpret_cast<void *>(&node_run_kernel<T, G, NV, W, 2>);
    return reinterpret_cast<void *>(&node_run_kernel<T, G, NV, W, 0>);
}

// Warp-wide rows (one or two vectors per lane) and narrow rows of one vector
// per lane in groups of 4, 8 or 16 lanes (each group with its own Y').
template <typename T, bool W>
void *pick_run(int g, int nv, int form) {
    if (nv == 2) return g == 32 ? pick_form<T, 32, 2, W>(form) : nullptr;
    if (nv != 1) return nullptr;
    switch (g) {
        case 32: return pick_form<T, 32, 1, W>(form);
        case 16: return pick_form<T, 16, 1, W>(form);
        case 8: return pick_form<T, 8, 1, W>(form);
        case 4: return pick_form<T, 4, 1, W>(form);
        default: return nullptr;
    }
}

// FP32 weighted and unweighted, FP64 unweighted (the weighted FP64 form stays
// on node_kernel: it serves the finite-difference reference only)
void *select_run(Elem e, int g, int nv, bool weighted, int form) {
    if (e == Elem::F64) return weighted ? nullptr : pick_run<double, false>(g, nv, form);
    if (e == Elem::F32) return weighted ? pick_run<float, true>(g, nv, form) : pick_run<float, false>(g, nv, form);
    return nullptr;
}

}  // namespace

int node_run_blocks_per_sm(Elem e, int g, int nv, bool weighted, int form, int threads, size_t smem) {
    return blocks_per_sm(select_run(e, g, nv, weighted, form), threads, smem);
}

cudaError_t launch_node_run(const NodeArgs &args, Elem e, int g, int nv, int form, int threads, size_t smem,
                            int grid_cap, cudaStream_t stream) {
    void *k = select_run(e, g, nv, args.weights != nullptr, form);
    if (!k || !args.runmap) return cudaErrorInvalidValue;
    const cudaError_t err = ensure_smem(k, threads, smem);
    if (err != cudaSuccess) return err;
    NodeArgs a = args;
    a.group_rows = 0;  // one task per warp
    const int64_t uvec = (int64_t)a.nb * a.ldp / (e == Elem::F64 ? 2 : 4);
    // packed arcs hold u * uvec in 28 bits (the zero row n included)
    if ((a.n + 1) * uvec >= (int64_t(1) << 28)) return cudaErrorInvalidValue;
    a.uvec = (unsigned)uvec;
    return launch_variant(k, a, 32, threads, smem, grid_cap, stream);
}

}  // namespace sg2v
