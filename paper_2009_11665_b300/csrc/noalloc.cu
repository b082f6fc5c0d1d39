// Allocation-free summation of per-vertex counts (sg2v_sum_counts_noalloc).
//
// Some callers cannot allocate device memory at the point where they need a
// total: serving loops whose device memory is reserved up front by their own
// allocator (a further allocation may fail or be forbidden there), and code
// that must not stall other streams (cudaMalloc and cudaFree synchronise the
// device).  This entry point sums per-vertex counts the caller already holds
// on the device into per-segment totals without any allocation: its scratch
// is a fixed file-scope device array that every GPU loading the library keeps
// until the process exits.
//
// The arithmetic is that of the library's root reduction: each value that is
// a non-negative integer below 2^128 is added exactly in 128-bit integers and
// the sum is rounded once to the nearest double; if any value is not such an
// integer the total is a compensated (two-sum) FP64 sum instead.  Block
// partials are combined in a fixed order, so results are reproducible.
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>

#include "sg2v_internal.h"

namespace {

constexpr int kChunks = 64;         // blocks (partial records) per segment
constexpr int kMaxSegments = 1024;  // segments per call
constexpr int kMaxDevices = 64;

struct Partial {
    unsigned long long lo, hi;  // exact 128-bit integer sum
    double s, c;                // compensated FP64 sum s + c
    unsigned flags;             // bit 0: a value was not an integer in [0, 2^128); bit 1: non-finite
    unsigned pad;
};

// The scratch: one partial record per (segment, chunk); 2.5 MiB.
static __device__ __align__(256) Partial g_scratch[kMaxSegments * kChunks];

__device__ __forceinline__ void two_sum(double a, double b, double &s, double &e) {
    s = a + b;
    const double bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

__device__ __forceinline__ void combine(Partial &x, const Partial &y) {
    // 128-bit add with the carry out of each step kept apart: the high word
    // takes y.hi plus the low word's carry (which itself wraps when y.hi is
    // 2^64 - 1), then x.hi; a carry out of either step means the sum reached
    // 2^128
    const unsigned long long lo = x.lo + y.lo;
    const unsigned long long c0 = lo < x.lo ? 1ull : 0ull;
    const unsigned long long t = y.hi + c0;
    const unsigned long long hi = x.hi + t;
    if ((t < c0) | (hi < x.hi)) x.flags |= 1u;
    x.hi = hi;
    x.lo = lo;
    double s, e;
    two_sum(x.s, y.s, s, e);
    x.c = x.c + y.c + e;
    x.s = s;
    x.flags |= y.flags;
}

__device__ __forceinline__ Partial from_value(double v) {
    Partial r;
    r.lo = r.hi = 0;
    r.s = v;
    r.c = 0.0;
    r.flags = 0;
    r.pad = 0;
    if (!isfinite(v)) {
        r.flags = 2u;
    } else if (v != floor(v) || v < 0.0 || v >= 0x1p128) {
        r.flags = 1u;
    } else if (v < 0x1p64) {
        r.lo = __double2ull_rz(v);
    } else {
        const double h = floor(v * 0x1p-64);
        r.hi = __double2ull_rz(h);
        r.lo = __double2ull_rz(v - h * 0x1p64);
    }
    return r;
}

__device__ __forceinline__ Partial shfl_xor(const Partial &x, int o) {
    Partial y;
    y.lo = __shfl_xor_sync(0xffffffffu, x.lo, o);
    y.hi = __shfl_xor_sync(0xffffffffu, x.hi, o);
    y.s = __shfl_xor_sync(0xffffffffu, x.s, o);
    y.c = __shfl_xor_sync(0xffffffffu, x.c, o);
    y.flags = __shfl_xor_sync(0xffffffffu, x.flags, o);
    y.pad = 0;
    return y;
}

// 128-bit unsigned integer to the nearest double (ties to even): the top 64
// significant bits keep a sticky bit for everything below them, so the one
// rounding of the 64-bit conversion is the correct rounding of the whole.
__device__ __forceinline__ double u128_to_double(unsigned long long hi, unsigned long long lo) {
    if (hi == 0) return __ull2double_rn(lo);
    const int shift = 64 - __clzll((long long)hi);  // bits of the value above the low 64, 1..64
    const unsigned long long top = shift == 64 ? hi : (hi << (64 - shift)) | (lo >> shift);
    const unsigned long long sticky = (shift == 64 ? lo : (lo << (64 - shift))) != 0ull ? 1ull : 0ull;
    return ldexp(__ull2double_rn(top | sticky), shift);
}

__global__ void noalloc_partial_kernel(const double *__restrict__ values, int64_t n, Partial *scratch) {
    __shared__ Partial red[32];
    const int seg = blockIdx.y, chunk = blockIdx.x;
    const int64_t per = (n + kChunks - 1) / kChunks;
    const int64_t lo = (int64_t)chunk * per;
    const int64_t hi = lo + per < n ? lo + per : n;
    Partial acc = from_value(0.0);
    for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) combine(acc, from_value(values[(int64_t)seg * n + i]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const Partial y = shfl_xor(acc, o);
        combine(acc, y);
    }
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        Partial t = red[0];
        for (int i = 1; i < (int)(blockDim.x >> 5); ++i) combine(t, red[i]);
        scratch[(int64_t)seg * kChunks + chunk] = t;  // every record read below is written here first
    }
}

__global__ void noalloc_final_kernel(const Partial *scratch, int nseg, double *totals) {
    const int seg = blockIdx.x * blockDim.x + threadIdx.x;
    if (seg >= nseg) return;
    Partial t = scratch[(int64_t)seg * kChunks];
    for (int i = 1; i < kChunks; ++i) combine(t, scratch[(int64_t)seg * kChunks + i]);
    totals[seg] = t.flags == 0 ? u128_to_double(t.hi, t.lo) : t.s + t.c;
}

std::mutex g_setup_mutex;
Partial *g_scratch_address[kMaxDevices] = {nullptr};

bool on_device(const void *p) {
    cudaPointerAttributes attr;
    if (cudaPointerGetAttributes(&attr, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return attr.type == cudaMemoryTypeDevice || attr.type == cudaMemoryTypeManaged;
}

}  // namespace

extern "C" sg2v_status sg2v_sum_counts_noalloc(const double *values, int64_t n, int32_t nseg, double *totals,
                                               sg2v_stream stream) {
    if (!values || !totals || n < 1 || nseg < 1) {
        sg2v::set_error("sg2v_sum_counts_noalloc: null pointer or empty size");
        return SG2V_ERR_INVALID_ARGUMENT;
    }
    if (nseg > kMaxSegments) {
        sg2v::set_error("sg2v_sum_counts_noalloc: nseg exceeds the fixed scratch limit of 1024 segments");
        return SG2V_ERR_INVALID_ARGUMENT;
    }
    if (!on_device(values) || !on_device(totals)) {
        sg2v::set_error("sg2v_sum_counts_noalloc: values and totals must be device memory");
        return SG2V_ERR_INVALID_ARGUMENT;
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        sg2v::set_error("sg2v_sum_counts_noalloc: no usable current device");
        return SG2V_ERR_CUDA;
    }
    Partial *scratch;
    {
        // once per device, with that device current: the host-side name of
        // the array is not a device address, so ask the runtime for it (the
        // address is kept for the life of the process: a device reset, which
        // recreates the module, invalidates it)
        std::lock_guard<std::mutex> lock(g_setup_mutex);
        if (!g_scratch_address[dev]) {
            void *p = nullptr;
            e = cudaGetSymbolAddress(&p, g_scratch);
            if (e != cudaSuccess) {
                sg2v::set_error(std::string("sg2v_sum_counts_noalloc: cudaGetSymbolAddress: ") + cudaGetErrorString(e));
                return SG2V_ERR_CUDA;
            }
            g_scratch_address[dev] = static_cast<Partial *>(p);
        }
        scratch = g_scratch_address[dev];
    }
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    noalloc_partial_kernel<<<dim3(kChunks, (unsigned)nseg), 256, 0, s>>>(values, n, scratch);
    noalloc_final_kernel<<<(nseg + 127) / 128, 128, 0, s>>>(scratch, nseg, totals);
    e = cudaGetLastError();
    if (e != cudaSuccess) {
        sg2v::set_error(std::string("sg2v_sum_counts_noalloc: launch: ") + cudaGetErrorString(e));
        return SG2V_ERR_CUDA;
    }
    return SG2V_OK;
}
