// Device helpers shared by the kernel translation units: vector and
// integer-table arithmetic, reductions, the expansion of per-colour
// accumulators into Y' and the eMA epilogues.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <type_traits>

#include "kernels.cuh"

namespace sg2v {

namespace {


constexpr unsigned kFull = 0xffffffffu;
#ifndef SG2V_U_NV1
#define SG2V_U_NV1 4
#endif
#ifndef SG2V_U_NV2
#define SG2V_U_NV2 2
#endif
#ifndef SG2V_PACKED
#define SG2V_PACKED 1
#endif
constexpr int kMaxHistColours = 16;

template <typename T>
struct Vec16;
template <>
struct Vec16<float> {
    using type = float4;
    static constexpr int n = 4;
    __device__ static float4 zero() { return make_float4(0.f, 0.f, 0.f, 0.f); }
#if SG2V_PACKED
    // packed FP32x2 arithmetic (sm_100 family): two instructions per float4
    __device__ static void add(float4 &a, const float4 &b) {
        const float2 lo = __fadd2_rn(make_float2(a.x, a.y), make_float2(b.x, b.y));
        const float2 hi = __fadd2_rn(make_float2(a.z, a.w), make_float2(b.z, b.w));
        a = make_float4(lo.x, lo.y, hi.x, hi.y);
    }
    __device__ static void fma(float4 &a, float w, const float4 &b) {
        const float2 ww = make_float2(w, w);
        const float2 lo = __ffma2_rn(ww, make_float2(b.x, b.y), make_float2(a.x, a.y));
        const float2 hi = __ffma2_rn(ww, make_float2(b.z, b.w), make_float2(a.z, a.w));
        a = make_float4(lo.x, lo.y, hi.x, hi.y);
    }
#else
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
#endif
    __device__ static void store(float *p, const float4 &a) {
        p[0] = a.x;
        p[1] = a.y;
        p[2] = a.z;
        p[3] = a.w;
    }
    __device__ static float4 shfl_xor(const float4 &a, int o) {
        return make_float4(__shfl_xor_sync(0xffffffffu, a.x, o), __shfl_xor_sync(0xffffffffu, a.y, o),
                           __shfl_xor_sync(0xffffffffu, a.z, o), __shfl_xor_sync(0xffffffffu, a.w, o));
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
    __device__ static double2 shfl_xor(const double2 &a, int o) {
        return make_double2(__shfl_xor_sync(0xffffffffu, a.x, o), __shfl_xor_sync(0xffffffffu, a.y, o));
    }
};

// Exact integer tables: unsigned 64-bit counts.  Every sum and product of
// the DP is an integer (Alg. 3 / 5 on an unweighted graph), so these tables
// are exact while each entry stays below 2^64; Ar<u64> reports every wrap.
using u64 = unsigned long long;

// Arithmetic of the table type with overflow accounting.  Floating-point
// types round and leave ovf alone; for unsigned 64-bit counts a carry out of
// bit 63 of a sum increments ovf and a product whose high 64 bits are not
// zero sets it, so ovf != 0 exactly when some result wrapped (a thread makes
// far fewer than 2^32 checked steps between two reports).
template <typename T>
struct Ar {
    static constexpr bool exact = false;
    __device__ static void add(T &a, T b, unsigned &) { a += b; }
    __device__ static void mad(T &acc, T a, T b, unsigned &) { acc = fma(a, b, acc); }
    __device__ static T twice(T a, unsigned &) { return T(2) * a; }
};
template <>
struct Ar<u64> {
    static constexpr bool exact = true;
    __device__ static void add(u64 &a, u64 b, unsigned &ovf) {
        asm("add.cc.u64 %0, %0, %2;\n\taddc.u32 %1, %1, 0;" : "+l"(a), "+r"(ovf) : "l"(b));
    }
    __device__ static void mad(u64 &acc, u64 a, u64 b, unsigned &ovf) {
        ovf |= __umul64hi(a, b) != 0ull ? 1u : 0u;
        add(acc, a * b, ovf);
    }
    __device__ static u64 twice(u64 a, unsigned &ovf) {
        ovf |= (unsigned)(a >> 63);
        return a << 1;
    }
};

template <>
struct Vec16<u64> {
    using type = ulonglong2;
    static constexpr int n = 2;
    __device__ static ulonglong2 zero() { return make_ulonglong2(0ull, 0ull); }
    __device__ static void add(ulonglong2 &a, const ulonglong2 &b) {
        a.x += b.x;
        a.y += b.y;
    }
    // integer tables count unweighted graphs only: w is 1
    __device__ static void fma(ulonglong2 &a, u64 w, const ulonglong2 &b) {
        a.x += w * b.x;
        a.y += w * b.y;
    }
    __device__ static void store(u64 *p, const ulonglong2 &a) {
        p[0] = a.x;
        p[1] = a.y;
    }
    __device__ static ulonglong2 shfl_xor(const ulonglong2 &a, int o) {
        return make_ulonglong2(__shfl_xor_sync(0xffffffffu, a.x, o), __shfl_xor_sync(0xffffffffu, a.y, o));
    }
};

// Unsigned 128-bit counts (two 64-bit words): exact to 2^128, for counts
// that pass 2^64 (tree10 on a graph of 2^24 edges reaches about 2^94).
struct alignas(16) u128 {
    u64 lo, hi;
    u128() = default;
    __host__ __device__ constexpr u128(u64 l, u64 h) : lo(l), hi(h) {}
    __host__ __device__ constexpr u128(int x) : lo((u64)(long long)x), hi(0) {}
    // (weights and exponent factors are 1 on the integer path)
    __host__ __device__ explicit u128(float x) : lo((u64)x), hi(0) {}
    __device__ u128 &operator+=(const u128 &b) {
        asm("add.cc.u64 %0, %0, %2;\n\taddc.u64 %1, %1, %3;" : "+l"(lo), "+l"(hi) : "l"(b.lo), "l"(b.hi));
        return *this;
    }
    __device__ u128 &operator*=(const u128 &b) {
        const u64 h = __umul64hi(lo, b.lo) + lo * b.hi + hi * b.lo;
        lo *= b.lo;
        hi = h;
        return *this;
    }
};
__device__ __forceinline__ u128 operator*(u128 a, const u128 &b) { return a *= b; }

// Shuffles, cache-global loads and atomic adds of 128-bit counts (the
// built-in overloads stay visible beside them).
using ::__shfl_sync;
using ::__shfl_xor_sync;
using ::__ldcg;
__device__ __forceinline__ u128 __shfl_sync(unsigned mask, const u128 &v, int src, int width = 32) {
    return u128(__shfl_sync(mask, v.lo, src, width), __shfl_sync(mask, v.hi, src, width));
}
__device__ __forceinline__ u128 __shfl_xor_sync(unsigned mask, const u128 &v, int o, int width = 32) {
    return u128(__shfl_xor_sync(mask, v.lo, o, width), __shfl_xor_sync(mask, v.hi, o, width));
}
__device__ __forceinline__ u128 __ldcg(const u128 *p) {
    const ulonglong2 v = __ldcg(reinterpret_cast<const ulonglong2 *>(p));
    return u128(v.x, v.y);
}

__device__ __forceinline__ double u128_to_double(unsigned long long hi, unsigned long long lo) {
    if (hi == 0) return __ull2double_rn(lo);
    const int shift = 64 - __clzll((long long)hi);  // 1..64
    const unsigned long long top = shift == 64 ? hi : (hi << (64 - shift)) | (lo >> shift);
    const unsigned long long sticky = (shift == 64 ? lo : (lo << (64 - shift))) != 0ull ? 1ull : 0ull;
    return ldexp(__ull2double_rn(top | sticky), shift);
}

template <>
struct Ar<u128> {
    static constexpr bool exact = true;
    // a += b; a carry out of bit 127 increments ovf
    __device__ static void add(u128 &a, const u128 &b, unsigned &ovf) {
        asm("add.cc.u64 %0, %0, %3;\n\taddc.cc.u64 %1, %1, %4;\n\taddc.u32 %2, %2, 0;"
            : "+l"(a.lo), "+l"(a.hi), "+r"(ovf)
            : "l"(b.lo), "l"(b.hi));
    }
    // acc += a * b; a product of 128 bits or more sets ovf
    __device__ static void mad(u128 &acc, const u128 &a, const u128 &b, unsigned &ovf) {
        const u64 c1 = a.lo * b.hi, c2 = a.hi * b.lo;
        const bool big = (a.hi != 0ull && b.hi != 0ull) || __umul64hi(a.lo, b.hi) != 0ull ||
                         __umul64hi(a.hi, b.lo) != 0ull;
        u128 p(a.lo * b.lo, __umul64hi(a.lo, b.lo));
        unsigned c = big ? 1u : 0u;
        asm("add.cc.u64 %0, %0, %2;\n\taddc.u32 %1, %1, 0;" : "+l"(p.hi), "+r"(c) : "l"(c1));
        asm("add.cc.u64 %0, %0, %2;\n\taddc.u32 %1, %1, 0;" : "+l"(p.hi), "+r"(c) : "l"(c2));
        ovf |= c;
        add(acc, p, ovf);
    }
    __device__ static u128 twice(const u128 &a, unsigned &ovf) {
        ovf |= (unsigned)(a.hi >> 63);
        return u128(a.lo << 1, (a.hi << 1) | (a.lo >> 63));
    }
};

template <>
struct Vec16<u128> {
    using type = u128;
    static constexpr int n = 1;
    __device__ static u128 zero() { return u128(0ull, 0ull); }
    __device__ static void add(u128 &a, const u128 &b) { a += b; }
    __device__ static void fma(u128 &a, const u128 &w, const u128 &b) { a += w * b; }
    __device__ static void store(u128 *p, const u128 &a) { *p = a; }
    __device__ static u128 shfl_xor(const u128 &a, int o) { return __shfl_xor_sync(0xffffffffu, a, o); }
};

// a += b for a 16-byte vector, with overflow accounting for integer tables.
template <typename T>
__device__ __forceinline__ void vadd(typename Vec16<T>::type &a, const typename Vec16<T>::type &b, unsigned &ovf) {
    if constexpr (Ar<T>::exact && Vec16<T>::n == 1) {
        Ar<T>::add(a, b, ovf);
    } else if constexpr (Ar<T>::exact) {
        Ar<T>::add(a.x, b.x, ovf);
        Ar<T>::add(a.y, b.y, ovf);
    } else {
        (void)ovf;
        Vec16<T>::add(a, b);
    }
}

// *p += x in global memory (partial rows of split rows), with overflow
// accounting for integer tables.
template <typename T>
__device__ __forceinline__ void atomic_add(T *p, T x, unsigned &ovf) {
    if constexpr (std::is_same<T, u128>::value) {
        // low word first; its carry goes into the high word's add, so the
        // 128-bit sum of all adds is exact in any order
        const u64 old_lo = atomicAdd(&p->lo, x.lo);
        const u64 c = old_lo + x.lo < old_lo ? 1ull : 0ull;
        const u64 add_hi = x.hi + c;
        if (add_hi < c) ovf |= 1u;
        const u64 old_hi = atomicAdd(&p->hi, add_hi);
        ovf |= old_hi + add_hi < old_hi ? 1u : 0u;
    } else if constexpr (Ar<T>::exact) {
        const T old = atomicAdd(p, x);
        ovf |= old + x < old ? 1u : 0u;
    } else {
        (void)ovf;
        atomicAdd(p, x);
    }
}

// Bit 1 of status word 0: a count left the range of the table type.
constexpr unsigned kStatusOverflow = 2u;

// Integer tables: a thread that saw a wrap raises the overflow status.
template <typename T>
__device__ __forceinline__ void report_ovf(unsigned *status, unsigned &ovf) {
    if constexpr (Ar<T>::exact) {
        if (ovf) {
            atomicOr(status, kStatusOverflow);
            ovf = 0;
        }
    } else {
        (void)status;
        (void)ovf;
    }
}

// Load of one 16-byte vector of a gathered table row (read-only path).
template <typename VT>
__device__ __forceinline__ VT ldg_row(const VT *p) {
    return __ldg(p);
}
template <>
__device__ __forceinline__ u128 ldg_row<u128>(const u128 *p) {
    const ulonglong2 v = __ldg(reinterpret_cast<const ulonglong2 *>(p));
    return u128(v.x, v.y);
}

// 2^d as a float for an exponent difference d <= 0 (0 below the normal range).
__device__ __forceinline__ float exp2_neg(int d) { return d < -126 ? 0.f : __int_as_float((d + 127) << 23); }

__device__ __forceinline__ int16_t clamp_exp(int e) {
    return (int16_t)(e > 32767 ? 32767 : (e < -32767 ? -32767 : e));
}

// A row's reference exponent; rows that gather nothing keep the pre-fill value.
__device__ __forceinline__ int row_eref(const NodeArgs &A, int64_t rowb) {
    const int e = A.Eref[rowb];
    return e < kEmptyRowExp ? kEmptyRowExp : e;
}

template <typename T>
__device__ __forceinline__ T warp_max(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(kFull, v, o));
    return v;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}

// Sum / maximum over an aligned group of G lanes (every lane of the warp
// takes part; each group gets its own result).
template <int G, typename T>
__device__ __forceinline__ T group_sum(T v) {
#pragma unroll
    for (int o = G >> 1; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}

template <int G, typename T>
__device__ __forceinline__ T group_sum_chk(T v, unsigned &ovf) {
#pragma unroll
    for (int o = G >> 1; o > 0; o >>= 1) Ar<T>::add(v, __shfl_xor_sync(kFull, v, o), ovf);
    return v;
}

template <int G, typename T>
__device__ __forceinline__ T group_max(T v) {
#pragma unroll
    for (int o = G >> 1; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(kFull, v, o));
    return v;
}

// Colour-compressed accumulation of one (row, colouring b) over arcs [e0, e1).
//
// Every table row u stores only the colour sets containing u's colour c_u
// (a count with u at the sub-template's root is zero otherwise), indexed by
// the remaining p-1 colours in the squeezed universe of c_u.  The SpMM is
// needed only for sets P without v's colour c_v, so arcs to neighbours of
// colour c_v are skipped, and the neighbour rows are summed per neighbour
// colour d into Z(d, .) (shared memory, private to the warp):
//   Y(v, P) = sum over d in P of Z(d, squeezed P - {d}).
// The warp splits into 32/G groups of G lanes; each group takes every
// (32/G)-th arc of a batch of 32 and owns a private copy of Z, and its lanes
// cover G*NV 16-byte vectors of the neighbour's compressed row (so narrow rows
// still fill a warp-wide load).  Copies are folded into copy 0 at the end.
template <typename T, int G, int NV, bool WEIGHTED, bool SCALED>
__device__ __forceinline__ void spmm_z(const NodeArgs &A, int v, int64_t e0, int64_t e1, int b, int cv, int eref,
                                       T *zbuf, int lane, unsigned &ovf) {
    constexpr bool FMA = WEIGHTED || SCALED;
    using V = Vec16<T>;
    using VT = typename V::type;
    constexpr int NG = 32 / G;
    constexpr int U = NV == 1 ? SG2V_U_NV1 : NV == 2 ? SG2V_U_NV2 : 2;  // arcs in flight per group and step
    const int grp = lane / G, gl = lane % G;
    const int kc = A.kc;
    const int wzp = A.wz_pad;  // = G * NV * V::n
    const int zlen = kc * wzp;
    VT *zv = reinterpret_cast<VT *>(zbuf);
    T *zg = zbuf + grp * zlen;
    static_assert(32 % (NG * U) == 0, "a step's arcs must stay inside one batch of 32");
    // FP64 adds are scarce on this part: there, arcs that read the zero row
    // skip their load and adds, and lanes past the row's last vector load
    // nothing.  FP32 loads stay unpredicated (measured faster): lanes past
    // the last vector read the next row or the table's padding into Z
    // columns that nothing reads.
    constexpr bool SKIP_ZERO = sizeof(T) >= 8;
    const int nvec = (A.Wz + V::n - 1) / V::n;
    bool qok[NV];
#pragma unroll
    for (int q = 0; q < NV; ++q) qok[q] = gl + G * q < nvec;
    bool qld[NV];  // FP32: lanes that load (all, or only those inside the row)
#pragma unroll
    for (int q = 0; q < NV; ++q) qld[q] = !A.pred_lanes || qok[q];
    // integer tables of odd width: the last vector's second element is row
    // padding that no kernel writes; it is cleared so that it adds no carry
    bool tail[NV];
#pragma unroll
    for (int q = 0; q < NV; ++q) tail[q] = Ar<T>::exact && V::n == 2 && (A.Wz & 1) && gl + G * q == nvec - 1;
    const int64_t uvec = (int64_t)A.nb * A.ldp / V::n;  // vectors between consecutive vertices' rows
    const VT *Mb = reinterpret_cast<const VT *>(static_cast<const T *>(A.Mp) + (int64_t)b * A.ldp) + gl;
    const int32_t *scol = A.scol + (int64_t)b * A.nnz;
    const int8_t *sclr = A.sclr + (int64_t)b * A.nnz;
    const float *sw = WEIGHTED ? A.sw + (int64_t)b * A.nnz : nullptr;
    const int16_t *Ep = SCALED ? A.Ep + b : nullptr;  // exponent of row (u, b) at Ep[u * nb]
    // the arcs come sorted by neighbour colour: each colour is one run, summed
    // in registers and written to Z(colour) when the run ends.  Each batch of
    // 32 arcs is compacted to the arcs that add something (a valid colour
    // other than v's own); slots past them read the table's zero row (vertex
    // n) into the current run.
    // A colour is one run per group, so its Z row is written once, without
    // reading it first; rows of colours with no arcs are zeroed at the end,
    // and the row of v's own colour (read by nothing) is left alone.
    VT run[NV];
#pragma unroll
    for (int q = 0; q < NV; ++q) run[q] = V::zero();
    int cur = -1;
    uint32_t seen = 0;  // colours whose Z row this group has written
    // narrow rows (G < 32): Z rows hold the row's vectors only (wzp / V::n
    // of them) and lanes past them write nothing; warp-wide rows keep the
    // warp's whole tile (measured faster without the guards)
    bool zok[NV];
#pragma unroll
    for (int q = 0; q < NV; ++q) zok[q] = G == 32 || gl + G * q < wzp / V::n;
    auto flush = [&](int c) {
        if (c != cv) {
            VT *zr = reinterpret_cast<VT *>(zg + c * wzp) + gl;
#pragma unroll
            for (int q = 0; q < NV; ++q)
                if (zok[q]) zr[G * q] = run[q];
            seen |= 1u << c;
        }
#pragma unroll
        for (int q = 0; q < NV; ++q) run[q] = V::zero();
    };
    const int zero_row = (int)A.n;
    for (int64_t base = e0; base < e1; base += 32) {
        const int cnt_in = (int)(e1 - base < 32 ? e1 - base : 32);
        const int c_in = lane < cnt_in ? (int)__ldg(sclr + base + lane) : -1;
        bool t_in = c_in >= 0 && c_in != cv;
        const int u_in = t_in ? __ldg(scol + base + lane) : zero_row;
        if (A.half_arcs && u_in >= v) t_in = false;
        // compact the batch to the arcs that add something (order kept, so
        // colour runs stay contiguous): lane j takes the j-th such arc
        const unsigned live_in = __ballot_sync(kFull, t_in);
        const int cnt = __popc(live_in);
        const bool t_l = lane < cnt;
        const int src = t_l ? (int)__fns(live_in, 0, lane + 1) : lane;
        int u_l = __shfl_sync(kFull, u_in, src);
        int c_l = __shfl_sync(kFull, c_in, src);
        // slots past the live arcs read the zero row into the batch's last
        // run, so a colour run that continues in the next batch is not cut
        const int c_last = __shfl_sync(kFull, c_l, cnt > 0 ? cnt - 1 : 0);
        if (!t_l) {
            u_l = zero_row;
            c_l = c_last;
        }
        T w_l = T(1);
        if (WEIGHTED) w_l = t_l ? T(__ldg(sw + base + src)) : T(0);
        int ep_l = eref;
        if (SCALED && t_l) ep_l = (int)__ldg(Ep + (int64_t)u_l * A.nb);
        for (int j0 = 0; j0 < cnt; j0 += NG * U) {
            VT x[U][NV];
            T w[U];
            int cr[U];
            bool live[U];
#pragma unroll
            for (int r = 0; r < U; ++r) {
                const int j = j0 + r * NG + grp;
                const int u = __shfl_sync(kFull, u_l, j);
                live[r] = !SKIP_ZERO || u != zero_row;
                cr[r] = __shfl_sync(kFull, c_l, j);
                w[r] = WEIGHTED ? __shfl_sync(kFull, w_l, j) : T(1);
                if (SCALED) {
                    // align the neighbour row's exponent to the row's reference
                    const int ep = __shfl_sync(kFull, ep_l, j);
                    w[r] *= T(exp2_neg(ep - eref));
                }
                const VT *row = Mb + (int64_t)u * uvec;
#pragma unroll
                for (int q = 0; q < NV; ++q) {
                    x[r][q] = (SKIP_ZERO ? (live[r] && qok[q]) : qld[q]) ? ldg_row(row + G * q) : V::zero();
                    if constexpr (Ar<T>::exact && V::n == 2)
                        if (tail[q]) x[r][q].y = 0;
                }
            }
#pragma unroll
            for (int r = 0; r < U; ++r) {
                if (!live[r]) continue;
                if (cr[r] != cur) {
                    if (cur >= 0) flush(cur);
                    cur = cr[r];
                }
#pragma unroll
                for (int q = 0; q < NV; ++q) {
                    if (FMA)
                        V::fma(run[q], w[r], x[r][q]);
                    else
                        vadd<T>(run[q], x[r][q], ovf);
                }
            }
        }
    }
    if (cur >= 0) flush(cur);
    for (int d = 0; d < kc; ++d) {
        if (!(seen >> d & 1u) && d != cv) {
            VT *zr = reinterpret_cast<VT *>(zg + d * wzp) + gl;
#pragma unroll
            for (int q = 0; q < NV; ++q)
                if (zok[q]) zr[G * q] = V::zero();
        }
    }
    __syncwarp();
    if (NG > 1) {
        // the copies' rows of v's own colour hold stale data: skipped
        const int own0 = cv * (wzp / V::n), own1 = own0 + wzp / V::n;
        for (int i = lane; i < zlen / V::n; i += 32) {
            if (i >= own0 && i < own1) continue;
            VT acc = zv[i];
#pragma unroll
            for (int g = 1; g < NG; ++g) vadd<T>(acc, zv[g * zlen / V::n + i], ovf);
            zv[i] = acc;
        }
    }
}

template <typename T>
__device__ __forceinline__ void hist_z_weighted(const NodeArgs &A, int64_t e0, int64_t e1, const int8_t *sclr,
                                                const float *sw, T *zbuf, int lane);

// Colour histogram of (row, colouring b): Z(d) = sum of w over arcs to
// neighbours of colour d (the passive child is a single vertex).
template <typename T, bool WEIGHTED>
__device__ __forceinline__ void hist_z(const NodeArgs &A, int64_t e0, int64_t e1, int b, T *zbuf, int lane) {
    const int8_t *sclr = A.sclr + (int64_t)b * A.nnz;
    if (!WEIGHTED) {
        // counts by warp ballots: every lane ends with every colour's count
        int cnt[kMaxHistColours];
#pragma unroll
        for (int c = 0; c < kMaxHistColours; ++c) cnt[c] = 0;
        for (int64_t base = e0; base < e1; base += 32) {
            const int64_t e = base + lane;
            const int c = e < e1 ? (int)__ldg(sclr + e) : -1;
#pragma unroll
            for (int q = 0; q < kMaxHistColours; ++q)
                if (q < A.kc) cnt[q] += __popc(__ballot_sync(kFull, c == q));
        }
        if (lane == 0) {
#pragma unroll
            for (int q = 0; q < kMaxHistColours; ++q)
                if (q < A.kc) zbuf[q] = T(cnt[q]);
        }
    } else {
        hist_z_weighted<T>(A, e0, e1, sclr, A.sw + (int64_t)b * A.nnz, zbuf, lane);
    }
}

template <typename T>
__device__ __forceinline__ void hist_z_weighted(const NodeArgs &A, int64_t e0, int64_t e1, const int8_t *sclr,
                                                const float *sw, T *zbuf, int lane) {
    T cnt[kMaxHistColours];
#pragma unroll
    for (int c = 0; c < kMaxHistColours; ++c) cnt[c] = T(0);
    for (int64_t e = e0 + lane; e < e1; e += 32) {
        const int c = __ldg(sclr + e);
        const T w = T(__ldg(sw + e));
#pragma unroll
        for (int q = 0; q < kMaxHistColours; ++q) cnt[q] += (c == q) ? w : T(0);
    }
#pragma unroll
    for (int q = 0; q < kMaxHistColours; ++q) {
        if (q < A.kc) {
            const T s = warp_sum(cnt[q]);
            if (lane == 0) zbuf[q] = s;
        }
    }
}

// Y'(j) = sum over the p offsets of set j of Z[offset] (ex: the table of the
// row's colour).  With stride 4 (2 <= p <= 4) the offsets of a set are one
// 8-byte load, with stride 8 (5 <= p <= 8) two, else they are read one by
// one (measured: one 16-byte load for p = 5 made the tree10 root slower).
template <typename T>
__device__ __forceinline__ T expand_set(const uint16_t *ex, int ps, int p, int j, const T *z, unsigned &ovf) {
    T s = T(0);
    const uint16_t *e = ex + (int64_t)j * ps;
    if (ps == 4) {
        const uint2 w = __ldg(reinterpret_cast<const uint2 *>(e));
        const uint32_t wd[2] = {w.x, w.y};
#pragma unroll
        for (int k = 0; k < 4; ++k)
            if (k < p) Ar<T>::add(s, z[(wd[k >> 1] >> (16 * (k & 1))) & 0xffffu], ovf);
    } else if (ps == 8) {
        const uint2 w0 = __ldg(reinterpret_cast<const uint2 *>(e));
        const uint2 w1 = __ldg(reinterpret_cast<const uint2 *>(e + 4));
        const uint32_t wd[4] = {w0.x, w0.y, w1.x, w1.y};
#pragma unroll
        for (int k = 0; k < 8; ++k)
            if (k < p) Ar<T>::add(s, z[(wd[k >> 1] >> (16 * (k & 1))) & 0xffffu], ovf);
    } else {
        for (int k = 0; k < p; ++k) Ar<T>::add(s, z[__ldg(e + k)], ovf);
    }
    return s;
}

// Y'(j) for the p-sets j of the squeezed universe of colour cv (the colour
// sets without cv the eMA needs), summed from Z into dst.
template <typename T>
__device__ __forceinline__ void expand_y(const NodeArgs &A, int cv, const T *zbuf, T *dst, int lane,
                                         unsigned &ovf) {
    const int p = A.p, wy = A.wy, ps = A.pstride;
    const uint16_t *ex = A.expand + (int64_t)cv * wy * ps;
    for (int j = lane; j < wy; j += 32) dst[j] = expand_set(ex, ps, p, j, zbuf, ovf);
}

// eMA (Eq. 1 in squeezed coordinates) of one row by NT threads (tid in
// [0, NT)).  The root needs only the row sum: every (set, split) product is
// one item, items are spread over all threads (consecutive threads read
// consecutive split words) and the per-thread partial sum is returned.  A
// thread that owns one output set of a non-root row walks its splits in
// order, so the split table's cache lines serve 32 consecutive steps.
template <typename T, int NT>
__device__ __forceinline__ T ema_root_partial(const NodeArgs &A, bool ok, const T *ybuf, const T *ma, int tid,
                                             unsigned &ovf) {
    T s = T(0);
    if (!ok) return s;
    if (A.a_leaf) {
        for (int j = tid; j < A.Ws; j += NT) Ar<T>::add(s, ybuf[j], ovf);
        return s;
    }
    const int total = A.Ws * A.nsplit;
    for (int p = tid; p < total; p += NT) {
        const uint32_t x = __ldg(A.splits + p);
        Ar<T>::mad(s, ma[x & 0xffffu], ybuf[x >> 16], ovf);
    }
    return s;
}

// Non-root rows: put(S, value) once per output set S.  Groups of L lanes
// (a power of two, L <= 32) share one set when there are fewer sets than
// threads, each lane taking every L-th split (adjacent words); with many
// sets L = 1.
template <typename T, int NT, typename F>
__device__ __forceinline__ void ema_rows(const NodeArgs &A, bool ok, const T *ybuf, const T *ma, int tid,
                                         unsigned &ovf, F &&put) {
    const int ws = A.Ws;
    if (A.a_leaf) {
        for (int S = tid; S < ws; S += NT) put(S, ok ? ybuf[S] : T(0));
        return;
    }
    const int ns = A.nsplit;
    int L = 32;
    while (L > 1 && NT / L < ws) L >>= 1;
    if (L == 1) {
        for (int S = tid; S < ws; S += NT) {
            T acc = T(0);
            if (ok) {
                const uint32_t *sp = A.splits + (int64_t)S * ns;
                for (int j = 0; j < ns; ++j) {
                    const uint32_t x = __ldg(sp + j);
                    Ar<T>::mad(acc, ma[x & 0xffffu], ybuf[x >> 16], ovf);
                }
            }
            put(S, acc);
        }
        return;
    }
    const int grp = tid / L, j0 = tid & (L - 1);
    for (int S0 = 0; S0 < ws; S0 += NT / L) {
        const int S = S0 + grp;
        T acc = T(0);
        if (ok && S < ws) {
            const uint32_t *sp = A.splits + (int64_t)S * ns;
            for (int j = j0; j < ns; j += L) {
                const uint32_t x = __ldg(sp + j);
                Ar<T>::mad(acc, ma[x & 0xffffu], ybuf[x >> 16], ovf);
            }
        }
        for (int o = L >> 1; o > 0; o >>= 1) Ar<T>::add(acc, __shfl_xor_sync(kFull, acc, o), ovf);
        if (j0 == 0 && S < ws) put(S, acc);
    }
}

// eMA in squeezed coordinates from Y' in ybuf:
//   M_s'(v, S') = sum over (a-1)-subsets A' of S' of M_a'(v, A') * Y'(S' - A'),
// or M_s' = Y' when the active child is a single vertex.  The root sums its
// row into root_out instead of storing it.  ok = false (a colour outside
// [0, kc), reported by the host) writes zeros.
template <typename T>
__device__ __forceinline__ void epilogue(const NodeArgs &A, int v, int b, bool ok, const T *ybuf, const T *ma,
                                         int lane, unsigned &ovf) {
    const int64_t rowb = (int64_t)v * A.nb + b;
    if (A.Yout) {
        T *yo = static_cast<T *>(A.Yout) + rowb * A.ldy;
        for (int j = lane; j < A.wy; j += 32) yo[j] = ok ? ybuf[j] : T(0);
    }
    if (A.root) {
        const T s = group_sum_chk<32>(ema_root_partial<T, 32>(A, ok, ybuf, ma, lane, ovf), ovf);
        if (lane == 0) static_cast<T *>(A.root_out)[(int64_t)b * A.n + v] = A.half_arcs ? Ar<T>::twice(s, ovf) : s;
        return;
    }
    T *out = static_cast<T *>(A.Ms) + rowb * A.ldt;
    const bool accumulate = A.accumulate != 0;
    ema_rows<T, 32>(A, ok, ybuf, ma, lane, ovf, [&](int S, T x) {
        if (accumulate) Ar<T>::add(x, out[S], ovf);
        out[S] = x;
    });
}

// Scaled FP32 eMA: outputs go to obuf first; the row is then normalised so
// its largest value lies in [1, 2) and its exponent is stored beside it.
// base is the exponent of the unnormalised outputs.  The root writes its
// row sum as a double with the exponent applied.
__device__ __forceinline__ void epilogue_scaled(const NodeArgs &A, int v, int b, bool ok, const float *ybuf,
                                                const float *ma, float *obuf, int base, int lane) {
    const int64_t rowb = (int64_t)v * A.nb + b;
    if (A.root) {
        unsigned ovf = 0;
        const float s = warp_sum(ema_root_partial<float, 32>(A, ok, ybuf, ma, lane, ovf));
        if (lane == 0) A.root_out_d[(int64_t)b * A.n + v] = ok ? ldexp((double)s, base + (A.half_arcs ? 1 : 0)) : 0.0;
        return;
    }
    float m = 0.f;
    unsigned ovf = 0;
    ema_rows<float, 32>(A, ok, ybuf, ma, lane, ovf, [&](int S, float x) {
        obuf[S] = x;
        m = fmaxf(m, x);
    });
    m = warp_max(m);
    const int em = m > 0.f ? ilogbf(m) : 0;
    __syncwarp();
    float *out = static_cast<float *>(A.Ms) + rowb * A.ldt;
    for (int j = lane; j < A.Ws; j += 32) out[j] = ldexpf(obuf[j], -em);
    if (lane == 0) A.Es[rowb] = m > 0.f ? clamp_exp(base + em) : kEmptyRowExp;
}

// Resident blocks per SM requested from the compiler (the register cap) for
// each shape; tuned on B300 (occupancy matters more than a few spills).
#ifndef SG2V_MINB_F32_NV2
#define SG2V_MINB_F32_NV2 5
#endif
#ifndef SG2V_MINB_F32_NV1
#define SG2V_MINB_F32_NV1 4
#endif
template <typename T, int NV>
struct MinBlocks {
    static constexpr int value =
        sizeof(T) == 4 ? (NV == 1 ? SG2V_MINB_F32_NV1 : NV == 2 ? SG2V_MINB_F32_NV2 : 2) : (NV == 1 ? 3 : 2);
};

}  // namespace

}  // namespace sg2v
