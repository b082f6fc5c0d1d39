// C ABI of the library: graph ingest, the DP executor and the reductions.
//
// The executor walks the planner's node list children-first (Alg. 2 "reverse
// order of partitioning"), launching one fused SpMM + eMA kernel per node
// (Alg. 5 inner loop), and finishes with the root reduction and finalCount
// of Alg. 1.  Count tables live in a library-owned stream-ordered memory pool
// and are released as soon as their last consumer has been launched.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <functional>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <tuple>
#include <vector>

#include "kernels.cuh"
#include "sg2v_internal.h"

namespace sg2v {

thread_local std::string g_last_error;

void set_error(const std::string &msg) { g_last_error = msg; }

namespace {

sg2v_status cuda_fail(cudaError_t e, const char *what) {
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        set_error(std::string(what) + ": out of device memory");
        return SG2V_ERR_OUT_OF_MEMORY;
    }
    set_error(std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")");
    return SG2V_ERR_CUDA;
}

#define SG2V_CUDA(call, what)                                   \
    do {                                                        \
        cudaError_t e_ = (call);                                \
        if (e_ != cudaSuccess) return cuda_fail(e_, what);      \
    } while (0)

bool is_device_pointer(const void *p) {
    if (!p) return false;
    cudaPointerAttributes attr;
    if (cudaPointerGetAttributes(&attr, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return attr.type == cudaMemoryTypeDevice || attr.type == cudaMemoryTypeManaged;
}

struct DeviceInfo {
    int sms = 0;
    int64_t l2_bytes = 0;
    cudaMemPool_t pool = nullptr;
};

std::mutex g_mutex;
std::map<int, DeviceInfo> g_devices;

sg2v_status device_info(int dev, DeviceInfo *out) {
    std::lock_guard<std::mutex> lock(g_mutex);
    auto it = g_devices.find(dev);
    if (it != g_devices.end()) {
        *out = it->second;
        return SG2V_OK;
    }
    DeviceInfo info;
    SG2V_CUDA(cudaDeviceGetAttribute(&info.sms, cudaDevAttrMultiProcessorCount, dev), "device attribute");
    int l2 = 0;
    SG2V_CUDA(cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev), "device attribute");
    info.l2_bytes = l2;
    cudaMemPoolProps props;
    std::memset(&props, 0, sizeof props);
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    SG2V_CUDA(cudaMemPoolCreate(&info.pool, &props), "memory pool");
    uint64_t keep = UINT64_MAX;  // keep freed blocks for the next call
    SG2V_CUDA(cudaMemPoolSetAttribute(info.pool, cudaMemPoolAttrReleaseThreshold, &keep), "memory pool");
    g_devices[dev] = info;
    *out = info;
    return SG2V_OK;
}

// Device copies of the colour-compressed expansion and split tables of node
// (t, a) for kc colours with Z rows of wz_pad elements (built once, kept).
struct DeviceTables {
    const uint16_t *expand = nullptr;  // [kc][wy][pstride]
    const uint32_t *expand32 = nullptr;  // [kc][wy][p] when offsets pass 16 bits (expand is then null)
    const uint32_t *splits = nullptr;
    const uint16_t *rootpair = nullptr;  // t = kc, a >= 2: rank(P') -> rank(A') of its one split
    int wy = 0, nsplit = 0, pstride = 1;
};

// Entries between consecutive sets of the device expansion table: the p
// offsets padded to 4 (2 <= p <= 4: one 8-byte load per set) or to 8
// (5 <= p <= 8: two).
int expand_stride(int p) { return (p >= 2 && p <= 4) ? 4 : ((p >= 5 && p <= 8) ? 8 : p); }
std::map<std::tuple<int, int, int, int, int>, DeviceTables> g_ctables;

sg2v_status device_tables(int dev, int kc, int t, int a, int wz_pad, DeviceTables *out) {
    std::lock_guard<std::mutex> lock(g_mutex);
    auto key = std::make_tuple(dev, kc, t, a, wz_pad);
    auto it = g_ctables.find(key);
    if (it != g_ctables.end()) {
        *out = it->second;
        return SG2V_OK;
    }
    CompressedTables tab;
    build_compressed_tables(kc, t, a, wz_pad, &tab);
    DeviceTables d;
    d.wy = tab.wy;
    d.nsplit = tab.nsplit;
    const int p = t - a, ps = expand_stride(p);
    d.pstride = ps;
    void *pe = nullptr, *ps_ = nullptr;
    const size_t bs = tab.splits.size() * sizeof(uint32_t);
    if ((int64_t)kc * wz_pad > 65536) {
        // Z offsets pass 16 bits: 32-bit offsets, one set after another
        const size_t be = tab.expand.size() * sizeof(uint32_t);
        SG2V_CUDA(cudaMalloc(&pe, std::max<size_t>(be, 16)), "table upload");
        SG2V_CUDA(cudaMemcpy(pe, tab.expand.data(), be, cudaMemcpyHostToDevice), "table upload");
        d.expand32 = static_cast<const uint32_t *>(pe);
        d.pstride = p;
    } else {
        std::vector<uint16_t> packed((size_t)kc * tab.wy * ps, 0);
        for (size_t set = 0; set < (size_t)kc * tab.wy; ++set)
            for (int k = 0; k < p; ++k) packed[set * ps + k] = (uint16_t)tab.expand[set * p + k];
        const size_t be = packed.size() * sizeof(uint16_t);
        SG2V_CUDA(cudaMalloc(&pe, std::max<size_t>(be, 16)), "table upload");
        SG2V_CUDA(cudaMemcpy(pe, packed.data(), be, cudaMemcpyHostToDevice), "table upload");
        d.expand = static_cast<const uint16_t *>(pe);
    }
    if (bs) {
        SG2V_CUDA(cudaMalloc(&ps_, bs), "table upload");
        SG2V_CUDA(cudaMemcpy(ps_, tab.splits.data(), bs, cudaMemcpyHostToDevice), "table upload");
    }
    d.splits = static_cast<const uint32_t *>(ps_);
    if (t == kc && a >= 2 && tab.nsplit == tab.wy && (int)tab.splits.size() == tab.nsplit) {
        // one output set: every p-set appears in exactly one split
        std::vector<uint16_t> pair((size_t)tab.wy, 0xffffu);
        for (uint32_t x : tab.splits) pair[x >> 16] = (uint16_t)(x & 0xffffu);
        bool perm = true;
        for (uint16_t q : pair) perm = perm && q != 0xffffu;
        if (perm) {
            void *pr = nullptr;
            SG2V_CUDA(cudaMalloc(&pr, pair.size() * sizeof(uint16_t)), "table upload");
            SG2V_CUDA(cudaMemcpy(pr, pair.data(), pair.size() * sizeof(uint16_t), cudaMemcpyHostToDevice),
                      "table upload");
            d.rootpair = static_cast<const uint16_t *>(pr);
        }
    }
    g_ctables[key] = d;
    *out = d;
    return SG2V_OK;
}

// Run map of node (t, a, p) for the run-scatter kernel: for the row's colour
// cv, a neighbour colour d and entry e of the neighbour's compressed row
// (the e-th (p-1)-subset Q' of d's squeezed universe, i.e. the p-set
// S = unsqueeze(Q', d) + {d}), the destination of that entry:
//   form 0 / 1: the colex rank of S in cv's squeezed p-sets (Y'),
//   form 2 (t = kc): the rank of the active set S' - S that completes S,
// or `sink` when S holds cv (and for d = cv, e >= C(kc-1, p-1)).
// Form 3 is the transposed SpMM of the backward pass: the gathered row is the
// neighbour's Ybar' (entry e: the e-th p-subset P of d's squeezed universe, a
// p-set without d) and the destination, for the row's colour cv, is the
// colex rank of P - {cv} in cv's squeezed (p-1)-sets (the compressed row of
// the passive table's gradient), or `sink` when P lacks cv.
// [kc][kc][wmap] 16-bit entries, cached per device.
std::map<std::tuple<int, int, int, int, int, int, int>, const uint16_t *> g_runmaps;

sg2v_status run_map(int dev, int kc, int t, int a, int form, int wmap, int sink, const uint16_t **out) {
    std::lock_guard<std::mutex> lock(g_mutex);
    const auto key = std::make_tuple(dev, kc, t, a, form, wmap, sink);
    auto it = g_runmaps.find(key);
    if (it != g_runmaps.end()) {
        *out = it->second;
        return SG2V_OK;
    }
    const int p = t - a;
    const bool transposed = form == 3;
    const int q_bits = transposed ? p : p - 1;  // colours of a gathered entry besides d
    const int wz = (int)binom(kc - 1, q_bits);
    const uint32_t full = (1u << (kc - 1)) - 1u;  // every colour of a squeezed universe
    std::vector<uint16_t> m((size_t)kc * kc * wmap, (uint16_t)sink);
    for (int d = 0; d < kc; ++d) {
        // the gathered row's sets in colex order: subsets by increasing mask
        std::vector<uint32_t> sets;
        sets.reserve((size_t)wz);
        for (uint32_t q = 0; q <= full; ++q)
            if (__builtin_popcount(q) == q_bits)
                sets.push_back(transposed ? unsqueeze_colour(q, d) : unsqueeze_colour(q, d) | (1u << d));
        for (int cv = 0; cv < kc; ++cv) {
            if (cv == d) continue;
            uint16_t *row = m.data() + ((size_t)cv * kc + d) * wmap;
            for (int e = 0; e < wz && e < wmap; ++e) {
                const uint32_t S = sets[(size_t)e];
                if (transposed) {
                    if (S >> cv & 1u) row[e] = (uint16_t)colex_rank(squeeze_colour(S & ~(1u << cv), cv));
                    continue;
                }
                if (S >> cv & 1u) continue;
                const uint32_t Sq = squeeze_colour(S, cv);
                row[e] = (uint16_t)(form == 2 ? colex_rank(full ^ Sq) : colex_rank(Sq));
            }
        }
    }
    void *dptr = nullptr;
    SG2V_CUDA(cudaMalloc(&dptr, m.size() * sizeof(uint16_t)), "table upload");
    SG2V_CUDA(cudaMemcpy(dptr, m.data(), m.size() * sizeof(uint16_t), cudaMemcpyHostToDevice), "table upload");
    g_runmaps[key] = static_cast<const uint16_t *>(dptr);
    *out = static_cast<const uint16_t *>(dptr);
    return SG2V_OK;
}

// Backward tables of a node (host copy for the counts, device copies for the
// kernels), built and uploaded once per device and node shape, kept for the
// life of the process like the run maps.
struct DeviceBackward {
    BackwardTables host;
    const uint32_t *ybar = nullptr, *mabar = nullptr, *arc = nullptr;
    const uint16_t *expand = nullptr;
};
std::map<std::tuple<int, int, int, int, int>, const DeviceBackward *> g_bwd_tables;

sg2v_status backward_tables(int dev, int kc, int t, int a, int wz_pad, const DeviceBackward **out) {
    std::lock_guard<std::mutex> lock(g_mutex);
    const auto key = std::make_tuple(dev, kc, t, a, wz_pad);
    auto it = g_bwd_tables.find(key);
    if (it != g_bwd_tables.end()) {
        *out = it->second;
        return SG2V_OK;
    }
    auto *d = new (std::nothrow) DeviceBackward();
    if (!d) return SG2V_ERR_OUT_OF_MEMORY;
    build_backward_tables(kc, t, a, wz_pad, &d->host);
    auto upload = [&](const void *h, size_t bytes, const void **dst) -> sg2v_status {
        void *p = nullptr;
        SG2V_CUDA(cudaMalloc(&p, std::max<size_t>(bytes, 16)), "table upload");
        if (bytes) SG2V_CUDA(cudaMemcpy(p, h, bytes, cudaMemcpyHostToDevice), "table upload");
        *dst = p;
        return SG2V_OK;
    };
    sg2v_status st;
    if ((st = upload(d->host.ybar.data(), d->host.ybar.size() * 4, (const void **)&d->ybar)) ||
        (st = upload(d->host.mabar.data(), d->host.mabar.size() * 4, (const void **)&d->mabar)) ||
        (st = upload(d->host.arc.data(), d->host.arc.size() * 4, (const void **)&d->arc)) ||
        (st = upload(d->host.expand.data(), d->host.expand.size() * 2, (const void **)&d->expand))) {
        cudaFree((void *)d->ybar);
        cudaFree((void *)d->mabar);
        cudaFree((void *)d->arc);
        cudaFree((void *)d->expand);
        delete d;
        return st;
    }
    g_bwd_tables[key] = d;
    *out = d;
    return SG2V_OK;
}

// ---- kernel timing records (measurement support)
struct ProfRecord {
    int64_t launches = 0;
    double total_ms = 0.0;
    double bytes = 0.0;  // summed over the launches
};
std::mutex g_prof_mutex;
bool g_prof_enabled = false;
std::map<std::string, ProfRecord> g_prof;
std::atomic<int64_t> g_launches{0};

// Event pairs of one call, folded into the records after its final sync.
struct CallTimer {
    bool on = false;
    bool count = true;  // false while a stream is being captured (replays count themselves)
    struct Item {
        std::string name;
        double bytes;
        cudaEvent_t a, b;
        int node;
    };
    std::vector<Item> items;
    cudaStream_t stream = nullptr;
    int open = -1;
    bool global = true;                   // add to the process-wide records
    std::vector<double> *node_ms = nullptr;  // per-node milliseconds (autotuning)
    CallTimer(cudaStream_t s) : stream(s) {
        std::lock_guard<std::mutex> lock(g_prof_mutex);
        on = g_prof_enabled;
    }
    void begin(const std::string &name, double bytes, int node = -1) {
        if (count) g_launches.fetch_add(1);
        if (!on) return;
        Item it{name, bytes, nullptr, nullptr, node};
        cudaEventCreate(&it.a);
        cudaEventCreate(&it.b);
        cudaEventRecord(it.a, stream);
        items.push_back(it);
        open = (int)items.size() - 1;
    }
    void end() {
        if (!on || open < 0) return;
        cudaEventRecord(items[open].b, stream);
        open = -1;
    }
    void count_extra(int n) {
        if (count) g_launches.fetch_add(n);
    }
    // call after the stream has been synchronised
    void collect() {
        if (!on) return;
        std::lock_guard<std::mutex> lock(g_prof_mutex);
        for (auto &it : items) {
            float ms = 0.f;
            if (cudaEventElapsedTime(&ms, it.a, it.b) == cudaSuccess) {
                if (node_ms && it.node >= 0 && it.node < (int)node_ms->size()) (*node_ms)[(size_t)it.node] += ms;
                if (!global) continue;
                ProfRecord &r = g_prof[it.name];
                r.launches += 1;
                r.total_ms += ms;
                r.bytes += it.bytes;
            }
        }
        cudaGetLastError();
    }
    ~CallTimer() {
        for (auto &it : items) {
            cudaEventDestroy(it.a);
            cudaEventDestroy(it.b);
        }
    }
};

int env_int(const char *name, int dflt) {
    const char *s = std::getenv(name);
    if (!s || !*s) return dflt;
    int v = std::atoi(s);
    return v > 0 ? v : dflt;
}

// The caller's allocator (sg2v_set_allocator), or none: the library's pool.
struct AllocHook {
    sg2v_alloc_fn alloc = nullptr;
    sg2v_free_fn free = nullptr;
    void *user = nullptr;
};
std::mutex g_hook_mutex;
AllocHook g_hook;

AllocHook current_hook() {
    std::lock_guard<std::mutex> lock(g_hook_mutex);
    return g_hook;
}

// Allocations of one call, returned on every exit path: from the caller's
// allocator when one is set (taken once, at the call's start), else from the
// library's stream-ordered pool.
thread_local int64_t g_last_peak_bytes = 0;

struct Workspace {
    cudaStream_t stream;
    cudaMemPool_t pool;
    std::vector<void *> live;
    AllocHook hook = current_hook();
    std::vector<size_t> sizes;  // of live blocks
    int64_t in_use = 0, peak = 0;
    ~Workspace() {
        for (void *p : live) give_back(p);
        g_last_peak_bytes = peak;
    }
    void give_back(void *p) {
        if (hook.alloc)
            hook.free(p, reinterpret_cast<sg2v_stream>(stream), hook.user);
        else
            cudaFreeAsync(p, stream);
    }
    sg2v_status alloc(void **p, size_t bytes) {
        *p = nullptr;
        if (bytes == 0) bytes = 16;
        if (hook.alloc) {
            *p = hook.alloc(bytes, reinterpret_cast<sg2v_stream>(stream), hook.user);
            if (!*p) {
                set_error("workspace allocation: the caller's allocator returned no memory");
                return SG2V_ERR_OUT_OF_MEMORY;
            }
        } else {
            cudaError_t e = cudaMallocFromPoolAsync(p, bytes, pool, stream);
            if (e != cudaSuccess) return cuda_fail(e, "workspace allocation");
        }
        live.push_back(*p);
        sizes.push_back(bytes);
        in_use += (int64_t)bytes;
        peak = std::max(peak, in_use);
        return SG2V_OK;
    }
    void release(void *p) {
        auto it = std::find(live.begin(), live.end(), p);
        if (it != live.end()) {
            give_back(p);
            const size_t k = (size_t)(it - live.begin());
            in_use -= (int64_t)sizes[k];
            sizes.erase(sizes.begin() + (int64_t)k);
            live.erase(it);
        }
    }
};

}  // namespace
}  // namespace sg2v

// Rows of at most this many arcs may run one per lane group (narrow rows).
constexpr int kShortTaskArcs = 64;

struct sg2v_graph {
    int device = 0;
    int64_t n = 0, nnz = 0, max_degree = 0;
    bool weighted = false;
    int64_t *row_ptr = nullptr;
    int32_t *col_idx = nullptr;
    float *weights = nullptr;
    int4 *tasks = nullptr;
    int64_t ntasks = 0;
    int32_t *heavy_chunks = nullptr;
    int64_t nheavy = 0;
    int chunk = 0;
    // column panels of the work list (1: none): rows longer than
    // kShortTaskArcs are cut where their neighbours cross into the next of
    // `panels` equal ranges of vertices, and tasks are ordered panel by panel
    int panels = 1;
    int64_t short_begin = 0;  // first task of at most kShortTaskArcs arcs (the rest, sorted by work, are too)
    int64_t small_begin = 0;  // first task of at most kSortSmallArcs arcs
    // isolated vertices: when the work list ends in the empty tasks of rows
    // [live_rows, n) (vertices numbered by decreasing degree put them there),
    // forward counting launches only tasks [0, live_tasks); else live_tasks =
    // ntasks and live_rows = n
    int64_t live_tasks = 0, live_rows = 0;
    int32_t *rev = nullptr;  // reverse arc of every arc, built on the first backward call
    // vertices relabelled by decreasing degree (unless SG2V_GRAPH_KEEP_ORDER):
    // the device CSR is in the new order; iperm[new] = the caller's vertex,
    // arcmap[new arc] = the caller's arc (null when the caller's order is kept)
    int32_t *iperm = nullptr;
    int32_t *arcmap = nullptr;
    // work-list variants (another chunk size) that share every array above
    // except tasks, heavy_chunks and rev; built on demand, owned here
    bool view = false;
    std::vector<sg2v_graph *> views;
};

namespace sg2v {
namespace {

void free_graph(sg2v_graph *g) {
    if (!g) return;
    if (g->view) {
        cudaFree(g->tasks);
        cudaFree(g->heavy_chunks);
        cudaFree(g->rev);
        delete g;
        return;
    }
    for (sg2v_graph *v : g->views) free_graph(v);
    cudaFree(g->row_ptr);
    cudaFree(g->col_idx);
    cudaFree(g->weights);
    cudaFree(g->tasks);
    cudaFree(g->heavy_chunks);
    cudaFree(g->rev);
    cudaFree(g->iperm);
    cudaFree(g->arcmap);
    delete g;
}

template <typename T>
sg2v_status host_copy(const T *src, int64_t count, std::vector<T> *dst) {
    dst->resize((size_t)count);
    if (count == 0) return SG2V_OK;
    if (is_device_pointer(src)) {
        SG2V_CUDA(cudaMemcpy(dst->data(), src, sizeof(T) * (size_t)count, cudaMemcpyDeviceToHost), "graph copy");
    } else {
        std::memcpy(dst->data(), src, sizeof(T) * (size_t)count);
    }
    return SG2V_OK;
}

sg2v_status validate_csr(int64_t n, int64_t nnz, const std::vector<int64_t> &rp, const std::vector<int32_t> &ci,
                         const std::vector<float> *w, bool full) {
    if (rp[0] != 0 || rp[n] != nnz) {
        set_error("row_ptr must start at 0 and end at nnz");
        return SG2V_ERR_INVALID_ARGUMENT;
    }
    for (int64_t i = 0; i < n; ++i)
        if (rp[i + 1] < rp[i]) {
            set_error("row_ptr is not monotone");
            return SG2V_ERR_INVALID_ARGUMENT;
        }
    // every column index in range first: the symmetry lookups below index
    // rows by column
    bool in_range = true;
#pragma omp parallel for schedule(static) reduction(&& : in_range)
    for (int64_t e = 0; e < nnz; ++e) in_range = in_range && ci[e] >= 0 && ci[e] < n;
    if (!in_range) {
        set_error("col_idx entry out of range");
        return SG2V_ERR_INVALID_ARGUMENT;
    }
    if (!full) return SG2V_OK;
    int bad = 0;  // 2: not simple, 3: asymmetric, 4: bad weight
#pragma omp parallel for schedule(dynamic, 4096) reduction(max : bad)
    for (int64_t i = 0; i < n; ++i) {
        for (int64_t e = rp[i]; e < rp[i + 1]; ++e) {
            int32_t j = ci[e];
            if (j == i || (e > rp[i] && ci[e - 1] >= j)) {
                bad = std::max(bad, 2);
                break;
            }
            const int32_t *b0 = ci.data() + rp[j], *b1 = ci.data() + rp[j + 1];
            const int32_t *hit = std::lower_bound(b0, b1, (int32_t)i);
            if (hit == b1 || *hit != i) {
                bad = std::max(bad, 3);
                break;
            }
            if (w) {
                float x = (*w)[e];
                if (!std::isfinite(x) || x < 0.f || (*w)[hit - ci.data()] != x) {
                    bad = std::max(bad, 4);
                    break;
                }
            }
        }
    }
    switch (bad) {
        case 2:
            set_error("graph has a self-loop, a repeated arc or an unsorted row");
            return SG2V_ERR_GRAPH_NOT_SIMPLE;
        case 3:
            set_error("CSR is not symmetric");
            return SG2V_ERR_GRAPH_NOT_SIMPLE;
        case 4:
            set_error("weights must be finite, non-negative and symmetric");
            return SG2V_ERR_GRAPH_NOT_SIMPLE;
        default:
            return SG2V_OK;
    }
}

// Work list: rows longer than `chunk` arcs are cut into chunk-sized tasks
// that share a scratch slot; all tasks are ordered by decreasing work.
void build_tasks(int64_t n, const std::vector<int64_t> &rp, int chunk, std::vector<int4> *tasks,
                 std::vector<int32_t> *heavy_chunks) {
    std::vector<int32_t> order((size_t)n);
    for (int64_t i = 0; i < n; ++i) order[(size_t)i] = (int32_t)i;
    std::stable_sort(order.begin(), order.end(),
                     [&](int32_t x, int32_t y) { return rp[x + 1] - rp[x] > rp[y + 1] - rp[y]; });
    tasks->clear();
    heavy_chunks->clear();
    std::vector<int4> light;
    light.reserve((size_t)n);
    for (int32_t v : order) {
        int64_t d = rp[v + 1] - rp[v];
        if (d > chunk) {
            int32_t slot = (int32_t)heavy_chunks->size();
            int32_t nc = (int32_t)((d + chunk - 1) / chunk);
            heavy_chunks->push_back(nc);
            for (int32_t c = 0; c < nc; ++c) {
                int64_t b = (int64_t)c * chunk, e = std::min<int64_t>(d, b + chunk);
                tasks->push_back(make_int4(v, slot, (int)(rp[v] + b), (int)(rp[v] + e)));
            }
        } else {
            light.push_back(make_int4(v, -1, (int)rp[v], (int)rp[v + 1]));
        }
    }
    tasks->insert(tasks->end(), light.begin(), light.end());
}

// Relabels the vertices by decreasing degree (ties keep the caller's order):
// the rows of the hubs, which most arcs gather, share cache lines and sit
// together in L2, and the work list (by decreasing work) walks the tables in
// address order.  Rows keep increasing column order.  iperm[new] = old;
// arcmap[new arc] = old arc; the weights follow their arcs.
void relabel_by_degree(int64_t n, std::vector<int64_t> &rp, std::vector<int32_t> &ci, std::vector<float> *w,
                       std::vector<int32_t> *iperm, std::vector<int32_t> *arcmap) {
    const int64_t nnz = rp[(size_t)n];
    iperm->resize((size_t)n);
    for (int64_t i = 0; i < n; ++i) (*iperm)[(size_t)i] = (int32_t)i;
    std::stable_sort(iperm->begin(), iperm->end(),
                     [&](int32_t x, int32_t y) { return rp[x + 1] - rp[x] > rp[y + 1] - rp[y]; });
    std::vector<int32_t> newid((size_t)n);
    for (int64_t i = 0; i < n; ++i) newid[(size_t)(*iperm)[(size_t)i]] = (int32_t)i;
    std::vector<int64_t> rp2((size_t)n + 1, 0);
    for (int64_t i = 0; i < n; ++i) {
        const int32_t o = (*iperm)[(size_t)i];
        rp2[(size_t)i + 1] = rp2[(size_t)i] + (rp[o + 1] - rp[o]);
    }
    std::vector<int32_t> ci2((size_t)nnz);
    arcmap->resize((size_t)nnz);
#pragma omp parallel
    {
        std::vector<std::pair<int32_t, int32_t>> row;
#pragma omp for schedule(dynamic, 1024)
        for (int64_t i = 0; i < n; ++i) {
            const int32_t o = (*iperm)[(size_t)i];
            row.clear();
            for (int64_t e = rp[o]; e < rp[o + 1]; ++e) row.emplace_back(newid[(size_t)ci[(size_t)e]], (int32_t)e);
            std::sort(row.begin(), row.end());
            int64_t k = rp2[(size_t)i];
            for (const auto &x : row) {
                ci2[(size_t)k] = x.first;
                (*arcmap)[(size_t)k] = x.second;
                ++k;
            }
        }
    }
    if (w) {
        std::vector<float> w2((size_t)nnz);
        for (int64_t e = 0; e < nnz; ++e) w2[(size_t)e] = (*w)[(size_t)(*arcmap)[(size_t)e]];
        w->swap(w2);
    }
    rp.swap(rp2);
    ci.swap(ci2);
}

struct CNode {
    int t, a, p;
    int active, passive;  // combined ids or kLeaf
    bool is_root;
    int last_use;
    std::string canon;    // AHU form of the rooted sub-template
};

// Launch shape of one node: gather width, Z layout, shared memory, block size.
struct Shape {
    int wz, grp, nv, wz_pad, zwords, ywords, mwords, owords, threads;
    size_t smem;
    int blocks_per_sm;
    bool rows = false;  // histogram node run 32 rows per warp (hist_rows_kernel)
    int npass = 1;      // CTA-wide rows: column tiles per row
    bool zglobal = false;  // CTA-wide rows: Z in global memory (too wide for shared memory)
    bool group = false; // narrow rows: short tasks one per lane group (node_group_kernel)
    int wthreads = 0, wbps = 0;  // the one-warp-per-row launch of the longer tasks of a group node
    size_t wsmem = 0;
    bool defer = false; // eMA in its own launch over blocks of rows (ema_rows_kernel)
    // run-scatter kernel (plain FP32 / FP64 tables) for the one-task-per-warp
    // launch: its run maps into Y' (forms 0 and 1) and into the active row
    // (form 2: root with t = kc), and its own launch shape
    bool run = false;
    // the forms this node can take (the autotuner picks among them) and the
    // launch shapes they need: the plain one-task-per-warp kernel, the
    // lane-group kernel for short rows, the 32-rows-per-warp histogram kernel
    bool can_run = false, can_group = false, can_rows = false, can_defer = false;
    int p_threads = 0, p_bps = 0, g_threads = 0, g_bps = 0, r_threads = 0, r_bps = 0;
    size_t p_smem = 0, g_smem = 0, r_smem = 0;
    const uint16_t *runmap_y = nullptr;
    const uint16_t *runmap_m = nullptr;
    int wmap = 0, mzero = 0;
    int run_ywords = 0, run_mwords = 0, run_threads = 0, run_bps = 0;
    size_t run_smem = 0;
    int64_t ldy = 0;    // Y' row stride of a deferred node
};

// Everything about a (graph, plans, batch, precision) request that does not
// depend on the colourings: the merged node list (sub-templates shared within
// and across plans), shapes and column tables.
struct Prepared {
    const sg2v_graph *g = nullptr;
    std::vector<const sg2v_plan *> plans;
    int kc = 0, nb = 0, dev = 0;
    bool fp64 = false;
    bool scaled = false;          // FP32 tables with per-row power-of-two exponents
    Elem elem = Elem::F32;        // table element type
    size_t esz = 4;
    int vecn = 4;
    int l2_stream = 1;            // run-scatter kernel: evict-first hints on data used once
    int64_t n = 0;
    DeviceInfo info;
    std::vector<CNode> nodes;
    std::vector<int> plan_root;   // combined root node of each plan (-1: single vertex)
    std::vector<int> root_plan;   // plan of each combined root node
    std::vector<Shape> shape;
    std::vector<DeviceTables> tabs;
    int64_t scratch_ld = 1;
    int auto_wave = 1;            // widest wave whose gathered table fits half of L2
    int64_t defer_words = 0;      // largest deferred node's Y' row stride (0: none)
    size_t zglobal_bytes = 0;     // global Z of CTA-wide rows that do not fit shared memory
};

// Sets a node's form and the launch shape it needs (only forms the node can
// take are set).
void apply_form(Shape &sh, bool group, bool rows, bool run_off, bool defer_off) {
    sh.group = group && sh.can_group;
    sh.rows = rows && sh.can_rows;
    if (sh.can_run) sh.run = !run_off;
    if (sh.can_defer) sh.defer = !defer_off;
    if (sh.rows) {
        sh.threads = sh.r_threads;
        sh.smem = sh.r_smem;
        sh.blocks_per_sm = sh.r_bps;
    } else if (sh.group) {
        sh.wthreads = sh.p_threads;
        sh.wsmem = sh.p_smem;
        sh.wbps = sh.p_bps;
        sh.threads = sh.g_threads;
        sh.smem = sh.g_smem;
        sh.blocks_per_sm = sh.g_bps;
    } else {
        sh.threads = sh.p_threads;
        sh.smem = sh.p_smem;
        sh.blocks_per_sm = sh.p_bps;
    }
}

const char *elem_name(const Prepared &P) {
    if (P.scaled) return "fp32s";
    if (P.elem == Elem::U128) return "u128";
    return P.elem == Elem::F64 ? "fp64" : (P.elem == Elem::U64 ? "u64" : "fp32");
}

sg2v_status prepare(const sg2v_graph *g, const sg2v_plan *const *plans, int32_t num_plans, int32_t B,
                    sg2v_precision precision, Prepared *P) {
    if (!g || !plans || num_plans < 1 || B < 1 ||
        (precision != SG2V_FP64 && precision != SG2V_FP32 && precision != SG2V_FP32_SCALED &&
         precision != SG2V_U64 && precision != SG2V_U128)) {
        set_error("invalid argument");
        return SG2V_ERR_INVALID_ARGUMENT;
    }
    if ((precision == SG2V_U64 || precision == SG2V_U128) && g->weights) {
        set_error("integer tables count unweighted graphs only");
        return SG2V_ERR_UNSUPPORTED;
    }
    const int kc = plans[0] ? plans[0]->kc : 0;
    for (int i = 0; i < num_plans; ++i)
        if (!plans[i] || plans[i]->kc != kc) {
            set_error("plans must be non-null and share num_colours");
            return SG2V_ERR_INVALID_ARGUMENT;
        }
    SG2V_CUDA(cudaGetDevice(&P->dev), "cudaGetDevice");
    if (P->dev != g->device) {
        set_error("graph lives on another device");
        return SG2V_ERR_INVALID_ARGUMENT;
    }
    sg2v_status st = device_info(P->dev, &P->info);
    if (st) return st;
    P->g = g;
    P->plans.assign(plans, plans + num_plans);
    P->kc = kc;
    P->nb = B;
    P->fp64 = precision == SG2V_FP64;
    P->scaled = precision == SG2V_FP32_SCALED;
    P->elem = P->fp64 ? Elem::F64
                      : (precision == SG2V_U64 ? Elem::U64 : (precision == SG2V_U128 ? Elem::U128 : Elem::F32));
    P->esz = P->elem == Elem::F32 ? 4 : (P->elem == Elem::U128 ? 16 : 8);
    P->vecn = (int)(16 / P->esz);
    {
        // SG2V_L2_STREAM=0: no evict-first hints in the run-scatter kernel
        const char *ls = std::getenv("SG2V_L2_STREAM");
        P->l2_stream = (ls && std::atoi(ls) == 0) ? 0 : 1;
    }
    P->n = g->n;
    P->plan_root.assign(num_plans, -1);
    std::map<std::string, int> shared;
    for (int pi = 0; pi < num_plans; ++pi) {
        const sg2v_plan *pl = plans[pi];
        std::vector<int> remap(pl->nodes.size(), -1);
        for (size_t i = 0; i < pl->nodes.size(); ++i) {
            const PlanNode &pn = pl->nodes[i];
            if (!pn.is_root) {
                auto it = shared.find(pn.canon);
                if (it != shared.end()) {
                    remap[i] = it->second;
                    continue;
                }
            }
            CNode c{pn.t, pn.a, pn.p, pn.active == kLeaf ? kLeaf : remap[pn.active],
                    pn.passive == kLeaf ? kLeaf : remap[pn.passive], pn.is_root, -1, pn.canon};
            P->nodes.push_back(c);
            remap[i] = (int)P->nodes.size() - 1;
            if (!pn.is_root) shared[pn.canon] = remap[i];
            if (pn.is_root) P->plan_root[pi] = remap[i];
        }
    }
    auto &nodes = P->nodes;
    P->root_plan.assign(nodes.size(), -1);
    for (int pi = 0; pi < num_plans; ++pi)
        if (P->plan_root[pi] >= 0) P->root_plan[P->plan_root[pi]] = pi;
    for (size_t i = 0; i < nodes.size(); ++i) {
        if (nodes[i].active != kLeaf) nodes[nodes[i].active].last_use = (int)i;
        if (nodes[i].passive != kLeaf) nodes[nodes[i].passive].last_use = (int)i;
    }
    P->shape.resize(nodes.size());
    P->tabs.resize(nodes.size());
    int64_t widest = 1;
    const int wide_min = env_int("SG2V_WIDE_MIN_WZ", 1 << 30);
    for (size_t i = 0; i < nodes.size(); ++i) {
        const CNode &c = nodes[i];
        Shape &sh = P->shape[i];
        const bool hist = c.p == 1;
        sh.wz = hist ? 1 : (int)binom(kc - 1, c.p - 1);
        sh.grp = 32;
        sh.nv = 1;
        if (!hist) node_shape(P->vecn, sh.wz, &sh.grp, &sh.nv);
        if (!hist && sh.grp != kWideLanes && sh.wz >= wide_min) {
            // rows at least SG2V_WIDE_MIN_WZ wide go to the CTA-per-row kernel
            sh.grp = kWideLanes;
            sh.nv = (sh.wz + kWideThreads * P->vecn - 1) / (kWideThreads * P->vecn);
        }
        if (sh.grp == kWideLanes) {
            // rows wider than the CTA's tile walk their arcs once per column tile
            const int nvec = (sh.wz + P->vecn - 1) / P->vecn;
            if (sh.nv == 0) sh.nv = 4;
            sh.npass = (nvec + kWideThreads * sh.nv - 1) / (kWideThreads * sh.nv);
        }
        if (sh.nv == 0) {
            set_error("passive table wider than this build's register tile");
            return SG2V_ERR_UNSUPPORTED;
        }
        if (!hist) widest = std::max<int64_t>(widest, (sh.wz + P->vecn - 1) / P->vecn * P->vecn);
        // Z rows: narrow rows (lane groups) and CTA-wide rows hold the row's
        // vectors only, warp-wide rows the whole tile of their lanes
        sh.wz_pad = hist ? 1
                         : (sh.grp != 32 ? (sh.wz + P->vecn - 1) / P->vecn * P->vecn : sh.grp * sh.nv * P->vecn);
        if ((int64_t)kc * sh.wz_pad > 65536 && sh.grp != kWideLanes) {
            set_error("per-colour accumulators of more than 65,536 elements outside the CTA-wide kernel");
            return SG2V_ERR_UNSUPPORTED;
        }
        sh.ywords = ((int)binom(kc - 1, c.p) + 3) / 4 * 4;
        sh.mwords = c.a == 1 ? 0 : ((int)binom(kc - 1, c.a - 1) + 3) / 4 * 4;
        sh.owords = P->scaled ? ((int)binom(kc - 1, c.t - 1) + 3) / 4 * 4 : 0;
        P->scratch_ld = std::max<int64_t>(P->scratch_ld, hist ? kc : (int64_t)kc * sh.wz_pad);
        if (sh.grp == kWideLanes) {
            // one CTA per row: Z, Y' and the active row once per CTA; Z goes to
            // global memory (one slot per resident CTA) when it does not fit
            sh.zwords = kc * sh.wz_pad;
            sh.threads = kWideThreads;
            sh.smem = (size_t)(sh.zwords + sh.ywords + sh.mwords + sh.owords) * P->esz;
            if (sh.smem > 220 * 1024) {
                sh.zglobal = true;
                sh.smem = (size_t)(sh.ywords + sh.mwords + sh.owords) * P->esz;
            }
        } else {
            sh.zwords = hist ? (kc + 3) / 4 * 4 : (32 / sh.grp) * kc * sh.wz_pad;
            sh.threads = kNodeThreads;
            const size_t per_warp = (size_t)(sh.zwords + sh.ywords + sh.mwords + sh.owords) * P->esz;
            while (sh.threads > 32 && (size_t)(sh.threads / 32) * per_warp > 200 * 1024) sh.threads /= 2;
            sh.smem = (size_t)(sh.threads / 32) * per_warp;
        }
        if (sh.smem > 227 * 1024) {
            set_error("per-colour accumulators exceed shared memory (column tiling not built)");
            return SG2V_ERR_UNSUPPORTED;
        }
        sh.blocks_per_sm =
            P->scaled ? node_blocks_per_sm_scaled(hist, sh.grp, sh.nv, g->weights != nullptr, sh.threads, sh.smem)
                      : node_blocks_per_sm(P->elem, hist, sh.grp, sh.nv, g->weights != nullptr, sh.threads, sh.smem);
        if (sh.zglobal)
            P->zglobal_bytes = std::max(P->zglobal_bytes, (size_t)P->info.sms * std::max(sh.blocks_per_sm, 1) *
                                                              (size_t)sh.zwords * P->esz);
        sh.p_threads = sh.threads;
        sh.p_smem = sh.smem;
        sh.p_bps = sh.blocks_per_sm;
        const char *group_env = std::getenv("SG2V_GROUP_ROWS");
        if (!hist && sh.grp < 32 && sh.nv == 1 && !(group_env && std::atoi(group_env) == 0)) {
            // narrow rows: every lane group takes its own row
            const size_t per_warp =
                (size_t)(32 / sh.grp) * (kc * sh.wz_pad + sh.ywords + sh.mwords + sh.owords) * P->esz;
            const int threads = kNodeThreads;
            const size_t smem = per_warp * (threads / 32);
            const int bps = smem <= 200 * 1024 ? (P->scaled ? node_blocks_per_sm_scaled(false, sh.grp, 1,
                                                                                        g->weights != nullptr,
                                                                                        threads, smem, true)
                                                            : node_blocks_per_sm(P->elem, false, sh.grp, 1,
                                                                                 g->weights != nullptr, threads, smem,
                                                                                 true))
                                               : 0;
            if (bps >= 1 && sh.p_bps >= 1) {
                sh.can_group = true;
                sh.g_threads = threads;
                sh.g_smem = smem;
                sh.g_bps = bps;
            }
        }
        const char *rows_env = std::getenv("SG2V_HIST_ROWS");
        if (hist && !g->weighted && !(rows_env && std::atoi(rows_env) == 0)) {
            // 32 rows per warp when the block's active rows fit shared memory
            // (unweighted graphs: with weights the one-warp-per-row kernel
            // measured faster)
            const size_t per_warp = (size_t)(kc * 32 + 32 * sh.mwords + sh.ywords + sh.owords) * P->esz;
            const int threads = kNodeThreads;
            const size_t smem = per_warp * (threads / 32);
            const int bps = smem <= 160 * 1024
                                ? hist_rows_blocks_per_sm(P->elem, P->scaled, g->weights != nullptr, threads, smem)
                                : 0;
            if (bps >= 1) {
                sh.can_rows = true;
                sh.r_threads = threads;
                sh.r_smem = smem;
                sh.r_bps = bps;
            }
        }
        // the default forms: lane groups for short narrow rows, 32 rows per
        // warp for histogram nodes (each measured faster on B300)
        apply_form(sh, sh.can_group, sh.can_rows, false, false);
        if (sh.blocks_per_sm < 1) {
            set_error("node kernel cannot be resident with its shared memory");
            return SG2V_ERR_UNSUPPORTED;
        }
        if ((st = device_tables(P->dev, kc, c.t, c.a, sh.wz_pad, &P->tabs[i]))) return st;
        // gathering nodes of plain FP32 / FP64 tables: the one-task-per-warp
        // launch uses the run-scatter kernel (SG2V_RUN_KERNEL=0 keeps the
        // per-colour accumulators of node_kernel); short tasks of narrow rows
        // stay one per lane group (node_group_kernel)
        const char *run_env = std::getenv("SG2V_RUN_KERNEL");
        const char *narrow_env = std::getenv("SG2V_RUN_NARROW");  // 0: warp-wide rows only
        const bool narrow_ok = !(narrow_env && std::atoi(narrow_env) == 0);
        // (the run kernel packs a neighbour's first table vector and its colour
        // into one 32-bit word, (u * vectors per vertex) << 4 | colour, the zero
        // row n included: (n + 1) x vectors per vertex below 2^28; checked here
        // for one colouring per row and again at each launch for its wave)
        const int64_t pvecs = (binom(kc - 1, c.p - 1) + P->vecn - 1) / P->vecn;  // one colouring per row
        if (!(run_env && std::atoi(run_env) == 0) && !hist && sh.grp != kWideLanes && !sh.rows &&
            (P->n + 1) * pvecs < (int64_t(1) << 28) &&
            (sh.grp == 32 || narrow_ok) &&
            (sh.nv == 1 || (sh.nv == 2 && sh.grp == 32)) && !P->scaled &&
            (P->elem == Elem::F32 || P->elem == Elem::F64)) {
            const int E = P->vecn;
            const int wy = (int)binom(kc - 1, c.p);
            const int wa = c.a == 1 ? 1 : (int)binom(kc - 1, c.a - 1);
            const int ybase = (wy + E - 1) / E * E, mbase = (wa + E - 1) / E * E;
            const int ywords = ybase + E;
            const int mwords = (c.a >= 2 || c.is_root) ? mbase + E : 0;
            const int threads = kNodeThreads;
            // per warp: a copy of Y' per lane group, the active row, the compacted arcs
            const size_t smem =
                (size_t)(threads / 32) * ((size_t)((32 / sh.grp) * ywords + mwords) * P->esz + kRunCompactBytes);
            const int form = (c.is_root && c.t == kc) ? 2 : ((c.a == 1 && !c.is_root) ? 1 : 0);
            const int bps =
                node_run_blocks_per_sm(P->elem, sh.grp, sh.nv, g->weights != nullptr, form, threads, smem);
            if (bps >= 1) {
                sh.run = sh.can_run = true;
                sh.wmap = sh.grp * sh.nv * E;
                sh.mzero = mbase;
                if ((st = run_map(P->dev, kc, c.t, c.a, 0, sh.wmap, ybase, &sh.runmap_y))) return st;
                if (form == 2 && (st = run_map(P->dev, kc, c.t, c.a, 2, sh.wmap, mbase, &sh.runmap_m))) return st;
                sh.run_ywords = ywords;
                sh.run_mwords = mwords;
                sh.run_threads = threads;
                sh.run_smem = smem;
                sh.run_bps = bps;
            }
        }
        // large eMA (many sets times many splits per row, root excepted): its own launch over
        // blocks of rows, so each split-table word serves several rows
        const char *defer_env = std::getenv("SG2V_DEFER_EMA");  // 0: never; else the least products per row
        const int64_t defer_min = defer_env ? std::atoll(defer_env) : 32768;
        const int64_t ema_work = binom(kc - 1, c.t - 1) * binom(c.t - 1, c.a - 1);
        if (!hist && c.a >= 2 && !c.is_root && defer_min > 0 && ema_work >= defer_min) {
            NodeArgs probe;
            std::memset(&probe, 0, sizeof probe);
            probe.wy = (int)binom(kc - 1, c.p);
            probe.Wa = (int)binom(kc - 1, c.a - 1);
            probe.Ws = (int)binom(kc - 1, c.t - 1);
            const size_t smem = ema_rows_smem(probe, P->elem, P->scaled);
            if (ema_rows_blocks_per_sm(P->elem, P->scaled, smem) >= 1) {
                sh.defer = sh.can_defer = true;
                sh.ldy = (probe.wy + P->vecn - 1) / P->vecn * P->vecn;
                P->defer_words = std::max<int64_t>(P->defer_words, sh.ldy);
            }
        }
    }
    const double per_colouring = (double)P->n * widest * P->esz;
    const int w = (int)std::floor(0.5 * P->info.l2_bytes / per_colouring);
    const int forced = env_int("SG2V_WAVE", 0);
    P->auto_wave = std::max(1, std::min(B, forced > 0 ? forced : w));
    return SG2V_OK;
}

// Device buffers of one run for a given wave width.
struct RunBuffers {
    int wave = 1;
    int32_t *scol = nullptr;
    int8_t *sclr = nullptr;       // 16 bytes into its allocation (sclr_base)
    int8_t *sclr_base = nullptr;
    float *sw = nullptr;
    void *scratch = nullptr;
    unsigned *counters = nullptr;
    size_t scratch_bytes = 0, counter_bytes = 0;
    std::vector<void *> rootbuf;  // per plan: [nb][n] table type
    std::vector<void *> table;    // per node: one wave's table (scaled: then its row exponents)
    std::vector<int64_t> ld;
    int32_t *eref = nullptr;      // scaled: [n][wave] reference exponents
    void *defer_y = nullptr;      // Y' rows of a deferred-eMA node: [n][wave][defer_words]
    void *zglobal = nullptr;      // global Z of CTA-wide rows: [resident CTAs][kc][wz_pad]
    int32_t *hcount = nullptr;    // neighbour counts per colour from the sort: [n][wave][hld]
    int hld = 0;
    unsigned *status = nullptr;   // [4]: bit 0 colour out of range
    int8_t *colp = nullptr;       // colourings in the graph's vertex order (relabelled graphs)
    double *ones = nullptr;       // [nb][n] ones for single-vertex templates
    int chunks = 1;
    // forward counting of a graph whose isolated vertices are rows
    // [live_rows, n): no task of theirs runs and no table row of theirs is
    // written or read (a gathered row belongs to a neighbour, an active row to
    // the task's own vertex); the root reduction counts them as zeros
    bool live = false;
    RootSum *partials = nullptr;  // [plans][nb][chunks]
    RootSum *sums = nullptr;      // [plans][nb]
};

// Where node tables come from: per-call pool allocations freed after their
// last consumer, or a session's fixed buffers.
struct TableSource {
    virtual ~TableSource() {}
    virtual sg2v_status get(size_t node, size_t bytes, void **p) = 0;
    virtual void done(size_t node) = 0;
};

int64_t table_ld(const Prepared &P, const CNode &c) {
    return (binom(P.kc - 1, c.t - 1) + P.vecn - 1) / P.vecn * P.vecn;
}

// A table that node kernels gather from has n + 1 vertex rows: row n (one
// row per colouring) is zero and takes the gathers of arcs that add nothing,
// and kGatherPad bytes after the rows cover loads of a whole register tile
// from the last row (a warp: at most 32 x 4 vectors of 16 bytes; a
// CTA-per-row kernel: 8 warps x 32 x 4 vectors).
constexpr size_t kGatherPad = 16384;

size_t gather_table_bytes(int64_t n, int wb, int64_t ld, size_t esz) {
    return (size_t)(n + 1) * wb * ld * esz + kGatherPad;
}

sg2v_status zero_gather_row(void *table, int64_t n, int wb, int64_t ld, size_t esz, cudaStream_t stream) {
    SG2V_CUDA(cudaMemsetAsync(static_cast<char *>(table) + (size_t)n * wb * ld * esz, 0, (size_t)wb * ld * esz, stream),
              "memset");
    return SG2V_OK;
}

// Bytes of one node's table for wb colourings; scaled tables carry one int16
// exponent per row after the values (from table_exp_offset).
size_t table_exp_offset(const Prepared &P, const CNode &c, int wb) {
    return (gather_table_bytes(P.n, wb, table_ld(P, c), P.esz) + 255) / 256 * 256;
}

size_t table_bytes(const Prepared &P, const CNode &c, int wb) {
    if (!P.scaled) return gather_table_bytes(P.n, wb, table_ld(P, c), P.esz);
    return table_exp_offset(P, c, wb) + (size_t)(P.n + 1) * wb * sizeof(int16_t);
}

int16_t *table_exps(const Prepared &P, const RunBuffers &R, int node, int wb) {
    return reinterpret_cast<int16_t *>(static_cast<char *>(R.table[node]) + table_exp_offset(P, P.nodes[node], wb));
}

// Bytes of a root buffer element: the table type, or double for scaled tables.
size_t root_esz(const Prepared &P) { return P.scaled ? sizeof(double) : P.esz; }

// Allocates the non-table buffers of a run from `alloc(bytes, &ptr)`.
bool sort_counts_used(const Prepared &P);
int sort_hist_node(const Prepared &P);

template <typename Alloc>
sg2v_status alloc_run(const Prepared &P, int wave, Alloc alloc, RunBuffers *R) {
    const sg2v_graph *g = P.g;
    sg2v_status st;
    R->wave = wave;
    if ((st = alloc((size_t)wave * g->nnz * sizeof(int32_t), (void **)&R->scol))) return st;
    // sorted colours, with 16 bytes on either side for aligned 16-byte reads
    if ((st = alloc((size_t)wave * g->nnz + 32, (void **)&R->sclr_base))) return st;
    R->sclr = R->sclr_base + 16;
    if (g->weighted && (st = alloc((size_t)wave * g->nnz * sizeof(float), (void **)&R->sw))) return st;
    R->scratch_bytes = (size_t)(g->nheavy * wave * P.scratch_ld) * P.esz;
    R->counter_bytes = (size_t)(g->nheavy * wave) * sizeof(unsigned);
    if (g->nheavy) {
        if ((st = alloc(R->scratch_bytes, &R->scratch))) return st;
        if ((st = alloc(R->counter_bytes, (void **)&R->counters))) return st;
    }
    if (P.scaled && (st = alloc((size_t)P.n * wave * sizeof(int32_t), (void **)&R->eref))) return st;
    if (P.defer_words && (st = alloc((size_t)P.n * wave * P.defer_words * P.esz, &R->defer_y))) return st;
    if (P.zglobal_bytes && (st = alloc(P.zglobal_bytes, &R->zglobal))) return st;
    if (sort_counts_used(P)) {
        R->hld = (P.kc + 3) / 4 * 4;
        if ((st = alloc((size_t)P.n * wave * R->hld * sizeof(int32_t), (void **)&R->hcount))) return st;
    }
    R->rootbuf.assign(P.plans.size(), nullptr);
    for (size_t pi = 0; pi < P.plans.size(); ++pi)
        if (P.plan_root[pi] >= 0 && (st = alloc((size_t)P.nb * P.n * root_esz(P), &R->rootbuf[pi]))) return st;
    R->table.assign(P.nodes.size(), nullptr);
    R->ld.assign(P.nodes.size(), 0);
    if ((st = alloc(16, (void **)&R->status))) return st;
    if (g->iperm && (st = alloc((size_t)P.nb * P.n, (void **)&R->colp))) return st;
    // about 4,096 values per block of the partial sums (enough blocks to fill the GPU)
    R->chunks = (int)std::max<int64_t>(1, std::min<int64_t>(1024, (P.n + 4095) / 4096));
    const size_t segs = P.plans.size() * (size_t)P.nb;
    if ((st = alloc(sizeof(RootSum) * segs * R->chunks, (void **)&R->partials))) return st;
    if ((st = alloc(sizeof(RootSum) * segs, (void **)&R->sums))) return st;
    return SG2V_OK;
}

// Kernel arguments of node i for colourings [b0, b0 + wb) (output table set by the caller).
NodeArgs node_args(const Prepared &P, const RunBuffers &R, size_t i, int b0, int wb, const int8_t *wcol) {
    const sg2v_graph *g = P.g;
    const CNode &c = P.nodes[i];
    const Shape &sh = P.shape[i];
    const int kc = P.kc;
    NodeArgs A;
    std::memset(&A, 0, sizeof A);
    A.row_ptr = g->row_ptr;
    A.col_idx = g->col_idx;
    A.weights = g->weights;
    A.tasks = g->tasks;
    A.ntasks = R.live ? g->live_tasks : g->ntasks;
    A.heavy_chunks = g->heavy_chunks;
    A.n = P.n;
    A.live_rows = R.live ? g->live_rows : P.n;
    A.nb = wb;
    A.colours = wcol;
    A.kc = kc;
    A.nnz = g->nnz;
    A.scol = R.scol;
    A.sclr = R.sclr;
    A.sw = R.sw;
    A.hist = c.p == 1;
    A.Wz = sh.wz;
    A.wz_pad = sh.wz_pad;
    A.zwords = sh.zwords;
    A.ywords = sh.ywords;
    A.mwords = sh.mwords;
    A.p = c.p;
    if (!A.hist) {
        A.Mp = R.table[c.passive];
        A.ldp = R.ld[c.passive];
    }
    A.a_leaf = c.a == 1;
    if (!A.a_leaf) {
        A.Ma = R.table[c.active];
        A.lda = R.ld[c.active];
        A.Wa = (int)binom(kc - 1, c.a - 1);
    }
    A.Ws = (int)binom(kc - 1, c.t - 1);
    A.expand = P.tabs[i].expand;
    A.expand32 = P.tabs[i].expand32;
    A.pstride = P.tabs[i].pstride;
    A.wy = P.tabs[i].wy;
    A.splits = P.tabs[i].splits;
    A.nsplit = P.tabs[i].nsplit;
    // the root's pairing form (warp-per-row kernel, plain tables)
    const char *pair_env = std::getenv("SG2V_ROOT_PAIRS");
    if (c.is_root && !P.scaled && !A.hist && sh.grp == 32 && !sh.group && !sh.defer && P.tabs[i].wy <= 128 &&
        !(pair_env && std::atoi(pair_env) == 0))
        A.rootpair = P.tabs[i].rootpair;
    A.root = c.is_root;
    if (c.is_root) {
        char *rb = static_cast<char *>(R.rootbuf[P.root_plan[i]]) + (size_t)b0 * P.n * root_esz(P);
        if (P.scaled)
            A.root_out_d = reinterpret_cast<double *>(rb);
        else
            A.root_out = rb;
    }
    A.group_rows = sh.group;
    {
        // FP32 gathers load only lanes inside the row (SG2V_PRED_LANES=0: every lane)
        const char *pl = std::getenv("SG2V_PRED_LANES");
        A.pred_lanes = (pl && std::atoi(pl) == 0) ? 0 : 1;
    }
    A.l2_stream = P.l2_stream;
    if (P.scaled) {
        A.scaled = 1;
        A.owords = sh.owords;
        A.Eref = R.eref;
        if (!A.hist) A.Ep = table_exps(P, R, c.passive, wb);
        if (!A.a_leaf) A.Ea = table_exps(P, R, c.active, wb);
    }
    A.scratch = R.scratch;
    A.scratch_ld = P.scratch_ld;
    A.counters = R.counters;
    A.status = R.status;
    A.npass = sh.npass;
    A.zglobal = sh.zglobal ? R.zglobal : nullptr;
    if (sh.rows && R.hcount) {
        A.hcount = R.hcount;
        A.hld = R.hld;
    }
    return A;
}

// Launches node i's one-task-per-warp work on the run-scatter kernel.
cudaError_t launch_run_node(const Prepared &P, size_t i, const NodeArgs &A, cudaStream_t stream) {
    const CNode &c = P.nodes[i];
    const Shape &sh = P.shape[i];
    NodeArgs R = A;
    int form = 0;
    if (A.root && c.t == P.kc && !A.Yout && !A.defer && sh.runmap_m)
        form = 2;
    else if (A.a_leaf && !A.root && !A.defer && !A.Yout && !A.accumulate)
        form = 1;
    R.runmap = form == 2 ? sh.runmap_m : sh.runmap_y;
    R.wmap = sh.wmap;
    R.mzero = sh.mzero;
    R.ywords = sh.run_ywords;
    R.mwords = sh.run_mwords;
    return launch_node_run(R, P.elem, sh.grp, sh.nv, form, sh.run_threads, sh.run_smem, P.info.sms * sh.run_bps,
                           stream);
}

// Launches the forward kernel of node i with the prepared shape.
// Whether the run-scatter kernel's packed arcs can address every gathered row
// of this launch's wave ((n + 1) x vectors per vertex below 2^28); a wider
// wave runs the per-colour-accumulator kernel instead.
bool run_fits(const Prepared &P, const NodeArgs &A) {
    return (P.n + 1) * ((int64_t)A.nb * A.ldp / P.vecn) < (int64_t(1) << 28);
}

cudaError_t launch_forward_node(const Prepared &P, size_t i, const NodeArgs &A, cudaStream_t stream) {
    const Shape &sh = P.shape[i];
    const int grid_cap = P.info.sms * sh.blocks_per_sm;
    const bool run = sh.run && run_fits(P, A);
    if (sh.rows) return launch_hist_rows(A, P.elem, P.scaled, sh.threads, sh.smem, grid_cap, stream);
    if (sh.group) {
        // the longer tasks (the front of the work list) one per warp, the short
        // ones one per lane group
        const int64_t split = P.g->short_begin;
        NodeArgs W = A;
        W.group_rows = 0;
        W.ntasks = split;
        cudaError_t e = run ? launch_run_node(P, i, W, stream)
                        : P.scaled ? launch_node_scaled(W, sh.grp, sh.nv, sh.wthreads, sh.wsmem,
                                                        P.info.sms * sh.wbps, stream)
                                   : launch_node(W, P.elem, sh.grp, sh.nv, sh.wthreads, sh.wsmem,
                                                 P.info.sms * sh.wbps, stream);
        if (e != cudaSuccess) return e;
        NodeArgs S = A;
        S.tasks = A.tasks + split;
        S.ntasks = A.ntasks - split;
        return P.scaled ? launch_node_scaled(S, sh.grp, sh.nv, sh.threads, sh.smem, grid_cap, stream)
                        : launch_node(S, P.elem, sh.grp, sh.nv, sh.threads, sh.smem, grid_cap, stream);
    }
    if (run) return launch_run_node(P, i, A, stream);
    if (P.scaled) return launch_node_scaled(A, sh.grp, sh.nv, sh.threads, sh.smem, grid_cap, stream);
    return launch_node(A, P.elem, sh.grp, sh.nv, sh.threads, sh.smem, grid_cap, stream);
}

// Enqueues the whole DP for colourings d_col ([nb][n], device) on `stream`:
// colour check, per wave the colour sort and one launch per node, then the
// root reductions into R.sums (and per-vertex doubles when pv != null).
// Nothing here synchronises, so the sequence can be captured in a CUDA graph.
// The node whose table the colour sort writes from its bucket counts: a
// non-root histogram node with two single-vertex children (t = 2) on an
// unweighted graph with plain tables (-1: none; SG2V_SORT_HIST=0 turns the
// fusion off).  Its children are leaves, so it is the first node to run.
// Whether the colour sort also writes the per-colour neighbour counts of
// every row for the histogram nodes that run 32 rows per warp (unweighted
// graphs; SG2V_SORT_COUNTS=0 keeps their own counting).
bool sort_counts_used(const Prepared &P) {
    const char *env = std::getenv("SG2V_SORT_COUNTS");
    if ((env && std::atoi(env) == 0) || P.g->weights) return false;
    const int fused = sort_hist_node(P);
    for (size_t i = 0; i < P.nodes.size(); ++i)
        if (P.shape[i].rows && (int)i != fused) return true;
    return false;
}

// The (2, 1, 1) node of a weighted graph with plain FP32 / FP64 tables: its
// table is summed from the colour-sorted arcs by its own small kernel
// (SG2V_SORT_HIST=0 keeps the node kernels); -1 when there is none.
int weighted_hist_node(const Prepared &P) {
    const char *env = std::getenv("SG2V_SORT_HIST");
    if ((env && std::atoi(env) == 0) || P.scaled || !P.g->weighted || !P.g->weights || P.kc > 16 ||
        !(P.elem == Elem::F32 || P.elem == Elem::F64))
        return -1;
    for (size_t i = 0; i < P.nodes.size(); ++i) {
        const CNode &c = P.nodes[i];
        if (c.t == 2 && c.a == 1 && c.p == 1 && !c.is_root) return (int)i;
    }
    return -1;
}

int sort_hist_node(const Prepared &P) {
    const char *env = std::getenv("SG2V_SORT_HIST");
    if ((env && std::atoi(env) == 0) || P.scaled || P.g->weights) return -1;
    for (size_t i = 0; i < P.nodes.size(); ++i) {
        const CNode &c = P.nodes[i];
        if (c.t == 2 && c.a == 1 && c.p == 1 && !c.is_root) return (int)i;
    }
    return -1;
}

sg2v_status enqueue(const Prepared &P, RunBuffers &R, const int8_t *d_col, double *pv, TableSource &src,
                    cudaStream_t stream, CallTimer &timer) {
    const sg2v_graph *g = P.g;
    const int64_t n = P.n;
    const int nb = P.nb, kc = P.kc, wave = R.wave;
    const size_t esz = P.esz;
    sg2v_status st;
    SG2V_CUDA(cudaMemsetAsync(R.status, 0, 16, stream), "memset");
    if (g->iperm) {
        // the caller's colourings into the graph's vertex order
        timer.count_extra(1);
        SG2V_CUDA(launch_gather_i8(d_col, R.colp, g->iperm, n, nb, stream), "colour permutation");
        d_col = R.colp;
    }
    timer.count_extra(1);
    SG2V_CUDA(launch_check_colours(d_col, (int64_t)nb * n, kc, R.status, stream), "colour check");
    const char *skip_env = std::getenv("SG2V_SKIP_EMPTY");
    R.live = !(skip_env && std::atoi(skip_env) == 0) && g->live_rows < n;
    const int64_t ntasks = R.live ? g->live_tasks : g->ntasks;
    const int64_t small_begin = std::min(g->small_begin, ntasks);
    const int64_t live_rows = R.live ? g->live_rows : n;
    const char *half_env = std::getenv("SG2V_HALF_ROOT");
    const bool half_root = !(half_env && std::atoi(half_env) == 0);
    const int fused = sort_hist_node(P);
    const int whist = weighted_hist_node(P);
    for (int b0 = 0; b0 < nb; b0 += wave) {
        const int wb = std::min(wave, nb - b0);
        const int8_t *wcol = d_col + (int64_t)b0 * n;
        SortHist hist{nullptr, 0, P.elem, nullptr, 0, nullptr};
        double hist_bytes = 0.0;
        if (R.hcount) {
            // neighbour counts per colour for the histogram nodes
            if (g->nheavy)  // chunks of split rows add into zeroed rows
                SG2V_CUDA(cudaMemsetAsync(R.hcount, 0, (size_t)n * wb * R.hld * sizeof(int32_t), stream), "memset");
            hist.hcount = R.hcount;
            hist.hld = R.hld;
            hist_bytes += (double)n * wb * kc * sizeof(int32_t);
        }
        if (fused >= 0) {
            // the (2, 1, 1) node's table comes from the sort's bucket counts
            const CNode &c = P.nodes[(size_t)fused];
            R.ld[(size_t)fused] = table_ld(P, c);
            if ((st = src.get((size_t)fused, table_bytes(P, c, wb), &R.table[(size_t)fused]))) return st;
            if ((st = zero_gather_row(R.table[(size_t)fused], n, wb, R.ld[(size_t)fused], esz, stream))) return st;
            if (g->nheavy)  // chunks of split rows add into zeroed rows
                SG2V_CUDA(cudaMemsetAsync(R.table[(size_t)fused], 0, (size_t)n * wb * R.ld[(size_t)fused] * esz, stream),
                          "memset");
            hist.out = R.table[(size_t)fused];
            hist.ld = R.ld[(size_t)fused];
            hist_bytes += (double)n * wb * (kc - 1) * esz;
        }
        timer.begin("colour_sort",
                    (double)wb * (8.0 * (n + 1) + g->nnz * (4.0 + 4.0 + 1.0 + (g->weighted ? 8.0 : 0.0))) + hist_bytes);
        SG2V_CUDA(launch_colour_sort(g->tasks, ntasks, small_begin, g->col_idx, g->weights, n, g->nnz, wcol, wb, kc,
                                     R.scol, R.sclr, R.sw, hist, P.info.sms, stream),
                  "colour sort");
        timer.end();
        if (small_begin > 0 && small_begin < ntasks) timer.count_extra(1);  // the small-task sort
        for (size_t i = 0; i < P.nodes.size(); ++i) {
            const CNode &c = P.nodes[i];
            const Shape &sh = P.shape[i];
            if ((int)i == fused) continue;  // written by the sort
            if ((int)i == whist) {
                // weighted (2, 1, 1): colour sums of the sorted arcs' weights
                R.ld[i] = table_ld(P, c);
                if ((st = src.get(i, table_bytes(P, c, wb), &R.table[i]))) return st;
                if ((st = zero_gather_row(R.table[i], n, wb, R.ld[i], esz, stream))) return st;
                if (g->nheavy)  // chunks of split rows add into zeroed rows
                    SG2V_CUDA(cudaMemsetAsync(R.table[i], 0, (size_t)n * wb * R.ld[i] * esz, stream), "memset");
                char name[64];
                std::snprintf(name, sizeof name, "node t=%d a=%d p=%d %s", c.t, c.a, c.p, elem_name(P));
                // algorithmic bytes: the sorted arcs' colours and weights, the
                // colouring and the work list read once, the table written once
                timer.begin(name,
                            (double)wb * g->nnz * 5.0 + (double)live_rows * wb * (1.0 + (kc - 1) * (double)esz) +
                                16.0 * ntasks,
                            (int)i);
                SG2V_CUDA(launch_weighted_hist(g->tasks, ntasks, small_begin, R.sclr, R.sw, g->nnz, wcol, n, wb, kc,
                                               R.table[i], R.ld[i], nullptr, 0, P.elem, P.info.sms, stream),
                          "weighted histogram");
                timer.end();
                continue;
            }
            NodeArgs A = node_args(P, R, i, b0, wb, wcol);
            if (!c.is_root) {
                R.ld[i] = table_ld(P, c);
                if ((st = src.get(i, table_bytes(P, c, wb), &R.table[i]))) return st;
                if ((st = zero_gather_row(R.table[i], n, wb, R.ld[i], esz, stream))) return st;
                A.Ms = R.table[i];
                A.ldt = R.ld[i];
                if (P.scaled) A.Es = table_exps(P, R, (int)i, wb);
            }
            A.scratch = R.scratch;
            A.scratch_ld = P.scratch_ld;
            A.counters = R.counters;
            A.status = R.status;
            // totals only and a root whose two children are one table: each
            // edge's contribution is counted once from its lower end, doubled
            A.half_arcs = c.is_root && c.active == c.passive && c.active != kLeaf && !pv && !A.hist &&
                          sh.grp != kWideLanes && half_root;
            if (g->nheavy) {
                SG2V_CUDA(cudaMemsetAsync(R.scratch, 0, R.scratch_bytes, stream), "memset");
                SG2V_CUDA(cudaMemsetAsync(R.counters, 0, R.counter_bytes, stream), "memset");
            }
            if (P.scaled && !A.hist) {
                // reference exponent of every row: the largest among the rows it gathers
                SG2V_CUDA(cudaMemsetAsync(R.eref, 0x80, (size_t)n * wb * sizeof(int32_t), stream), "memset");
                timer.begin("eref", (double)wb * (g->nnz * 5.0 + live_rows * 6.0) + 16.0 * ntasks);
                SG2V_CUDA(launch_eref(g->tasks, ntasks, R.scol, R.sclr, wcol, n, g->nnz, wb, kc, A.Ep, R.eref,
                                      P.info.sms, stream),
                          "eref");
                timer.end();
            }
            {
                // algorithmic bytes: each input table, the sorted arc list
                // (neighbour, its colour, weight) and the colouring read once,
                // the output written once (rows of isolated vertices, when
                // skipped, are neither read nor written)
                const double rows = (double)live_rows * wb;
                double bytes = 8.0 * (n + 1) + (double)wb * g->nnz * (5.0 + (g->weighted ? 4.0 : 0.0));
                bytes += rows;  // colours
                if (!A.hist) bytes += rows * A.Wz * esz;
                if (!A.a_leaf && !(c.active == c.passive && !A.hist)) bytes += rows * binom(kc - 1, c.a - 1) * esz;
                bytes += c.is_root ? rows * esz : rows * A.Ws * esz;
                if (P.scaled) bytes += rows * (A.hist ? 2.0 : 6.0) + (A.a_leaf ? 0.0 : rows * 2.0);
                char name[64];
                std::snprintf(name, sizeof name, "node t=%d a=%d p=%d %s", c.t, c.a, c.p,
                              elem_name(P));
                timer.begin(name, bytes, (int)i);
            }
            if (sh.defer) {
                A.defer = 1;
                A.Yout = R.defer_y;
                A.ldy = sh.ldy;
            }
            SG2V_CUDA(launch_forward_node(P, i, A, stream), "node kernel launch");
            timer.end();
            if (sh.group) timer.count_extra(1);  // short and long tasks launch apart
            if (sh.defer) {
                const double rows = (double)live_rows * wb;
                char name[64];
                std::snprintf(name, sizeof name, "ema t=%d a=%d p=%d %s", c.t, c.a, c.p,
                              elem_name(P));
                timer.begin(name, rows * esz * (double)(sh.ldy + binom(kc - 1, c.a - 1) + A.Ws), (int)i);
                SG2V_CUDA(launch_ema_rows(A, P.elem, P.scaled, P.info.sms, stream), "eMA launch");
                timer.end();
            }
            if (c.active != kLeaf && P.nodes[c.active].last_use == (int)i) src.done(c.active);
            if (c.passive != kLeaf && P.nodes[c.passive].last_use == (int)i && c.passive != c.active)
                src.done(c.passive);
        }
    }
    for (size_t pi = 0; pi < P.plans.size(); ++pi) {
        double *pvp = pv ? pv + pi * (size_t)nb * n : nullptr;
        const void *vals = P.plan_root[pi] >= 0 ? R.rootbuf[pi] : R.ones;
        // root values: the table type, doubles for scaled tables and single-vertex plans
        const Elem ve = P.plan_root[pi] >= 0 ? (P.scaled ? Elem::F64 : P.elem) : Elem::F64;
        // (a single-vertex template counts every vertex, isolated ones too)
        const int64_t live = P.plan_root[pi] >= 0 ? live_rows : n;
        timer.begin("root_reduce", (double)nb * live * (ve == Elem::F32 ? 4 : (ve == Elem::U128 ? 16 : 8)) +
                                       (pvp ? (double)nb * n * 8 : 0.0));
        timer.count_extra(1);
        SG2V_CUDA(launch_root_reduce(vals, ve, n, live, nb, pvp, g->iperm, R.partials + pi * (size_t)nb * R.chunks,
                                     R.chunks, R.sums + pi * (size_t)nb, stream),
                  "root reduction");
        timer.end();
    }
    return SG2V_OK;
}

bool needs_ones(const Prepared &P) {
    for (int r : P.plan_root)
        if (r < 0) return true;
    return false;
}

}  // namespace
}  // namespace sg2v

struct sg2v_session {
    sg2v::Prepared P;
    sg2v::RunBuffers R;
    uint32_t flags = 0;
    sg2v::AllocHook hook;       // the caller's allocator at creation (or none)
    std::vector<void *> owned;  // everything allocated here
    std::vector<void *> owned_tables;
    int8_t *colours = nullptr;  // [nb][n] staging
    double *pv = nullptr;       // [plans][nb][n]
    double *totals = nullptr, *estimates = nullptr;  // [plans][nb]
    double *scale = nullptr;    // [2][plans] hi, lo
    cudaGraphExec_t exec = nullptr;
    cudaStream_t capture = nullptr;  // private stream the graph is recorded on (any stream may replay it)
    bool tuned = false;
    int64_t launches_per_run = 0;
    const sg2v_graph *base = nullptr;  // the caller's graph (P.g may be a work-list variant of it)
};

namespace sg2v {
namespace {

// Session buffers come from the caller's allocator when one was set at
// creation (on the legacy default stream, synchronised), else cudaMalloc.
sg2v_status session_malloc(sg2v_session *S, size_t bytes, void **p) {
    bytes = std::max<size_t>(bytes, 16);
    if (S->hook.alloc) {
        *p = S->hook.alloc(bytes, nullptr, S->hook.user);
        if (!*p) {
            set_error("session allocation: the caller's allocator returned no memory");
            return SG2V_ERR_OUT_OF_MEMORY;
        }
        return SG2V_OK;
    }
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) return cuda_fail(e, "session allocation");
    return SG2V_OK;
}

void session_mfree(sg2v_session *S, void *p) {
    if (S->hook.alloc) {
        cudaDeviceSynchronize();  // no replay may still use it
        S->hook.free(p, nullptr, S->hook.user);
    } else {
        cudaFree(p);
    }
}

void session_free_tables(sg2v_session *S) {
    for (void *p : S->owned_tables) session_mfree(S, p);
    S->owned_tables.clear();
    S->R.table.assign(S->P.nodes.size(), nullptr);
}

void session_free(sg2v_session *S) {
    if (!S) return;
    if (S->exec) cudaGraphExecDestroy(S->exec);
    if (S->capture) cudaStreamDestroy(S->capture);
    session_free_tables(S);
    for (void *p : S->owned) session_mfree(S, p);
    delete S;
}

// (Re)allocates the wave-dependent buffers of a session for `wave`.
sg2v_status session_alloc_wave(sg2v_session *S, int wave) {
    const Prepared &P = S->P;
    // wave-independent buffers (root outputs, reductions) are reused when present
    sg2v_status st;
    auto alloc = [&](size_t bytes, void **p) -> sg2v_status {
        sg2v_status s2 = session_malloc(S, bytes, p);
        if (s2) return s2;
        S->owned.push_back(*p);
        return SG2V_OK;
    };
    // wave-dependent: sorted arcs, split-row scratch, tables
    for (void *p : {(void *)S->R.scol, (void *)S->R.sclr_base, (void *)S->R.sw, S->R.scratch, (void *)S->R.counters,
                    (void *)S->R.eref, S->R.defer_y, (void *)S->R.hcount}) {
        if (!p) continue;
        auto it = std::find(S->owned.begin(), S->owned.end(), p);
        if (it != S->owned.end()) {
            session_mfree(S, p);
            S->owned.erase(it);
        }
    }
    const sg2v_graph *g = P.g;
    RunBuffers &R = S->R;
    R.wave = wave;
    R.scol = nullptr;
    R.sclr = nullptr;
    R.sclr_base = nullptr;
    R.sw = nullptr;
    R.scratch = nullptr;
    R.counters = nullptr;
    R.eref = nullptr;
    R.defer_y = nullptr;
    R.hcount = nullptr;
    if ((st = alloc((size_t)wave * g->nnz * sizeof(int32_t), (void **)&R.scol))) return st;
    if (sort_counts_used(P)) {
        R.hld = (P.kc + 3) / 4 * 4;
        if ((st = alloc((size_t)P.n * wave * R.hld * sizeof(int32_t), (void **)&R.hcount))) return st;
    }
    if (P.scaled && (st = alloc((size_t)P.n * wave * sizeof(int32_t), (void **)&R.eref))) return st;
    if (P.defer_words && (st = alloc((size_t)P.n * wave * P.defer_words * P.esz, &R.defer_y))) return st;
    if ((st = alloc((size_t)wave * g->nnz + 32, (void **)&R.sclr_base))) return st;
    R.sclr = R.sclr_base + 16;
    if (g->weighted && (st = alloc((size_t)wave * g->nnz * sizeof(float), (void **)&R.sw))) return st;
    R.scratch_bytes = (size_t)(g->nheavy * wave * P.scratch_ld) * P.esz;
    R.counter_bytes = (size_t)(g->nheavy * wave) * sizeof(unsigned);
    if (g->nheavy) {
        if ((st = alloc(R.scratch_bytes, &R.scratch))) return st;
        if ((st = alloc(R.counter_bytes, (void **)&R.counters))) return st;
    }
    session_free_tables(S);
    for (size_t i = 0; i < P.nodes.size(); ++i) {
        if (P.nodes[i].is_root) continue;
        R.ld[i] = table_ld(P, P.nodes[i]);
        void *t = nullptr;
        if ((st = session_malloc(S, table_bytes(P, P.nodes[i], wave), &t))) return st;
        S->owned_tables.push_back(t);
        R.table[i] = t;
    }
    return SG2V_OK;
}

struct FixedTables : TableSource {
    std::vector<void *> &table;
    explicit FixedTables(std::vector<void *> &t) : table(t) {}
    sg2v_status get(size_t i, size_t, void **p) override {
        *p = table[i];
        return SG2V_OK;
    }
    void done(size_t) override {}
};

// One run of the session's sequence on stream (no synchronisation).
sg2v_status session_enqueue(sg2v_session *S, cudaStream_t stream, bool timed, bool capturing = false,
                            std::vector<double> *node_ms = nullptr) {
    CallTimer timer(stream);
    if (!timed) timer.on = false;
    if (capturing) timer.count = false;
    if (node_ms) {
        // autotuning: per-node times only, nothing in the process-wide records
        timer.on = true;
        timer.global = false;
        timer.node_ms = node_ms;
    }
    FixedTables src(S->R.table);
    sg2v_status st = enqueue(S->P, S->R, S->colours, S->pv, src, stream, timer);
    if (st) return st;
    const int nseg = (int)S->P.plans.size() * S->P.nb;
    SG2V_CUDA(launch_finalize(S->R.sums, nseg, S->P.nb, S->scale, S->scale + S->P.plans.size(), S->totals,
                              S->estimates, S->R.status, stream),
              "finalize");
    if (timed || node_ms) {
        cudaError_t e = cudaStreamSynchronize(stream);
        if (e != cudaSuccess) return cuda_fail(e, "stream synchronize");
        timer.collect();
    }
    return SG2V_OK;
}

// ---- autotuning of the node kernels' forms
//
// Every node may take a few forms (Shape::can_*): the run-scatter kernel or
// per-colour accumulators (node_kernel), lane groups for short narrow rows
// or one row per warp, 32 histogram rows per warp or one, the eMA in its own
// launch or in the gather's epilogue.  The first run of an autotuning
// session times, besides the default, each single change of every node's
// form (all nodes changed at once, one configuration per run: the node
// launches are independent, so their CUDA-event times separate) and keeps
// each node's fastest form.  Choices are cached by (graph statistics,
// colours, node shape, table type, wave) in the JSON file named by
// SG2V_TUNE_CACHE, when set, so that later sessions skip the timing.

struct Form {
    bool group, rows, run_off, defer_off;
};

std::vector<Form> form_alternatives(const Shape &sh) {
    const Form d{sh.group, sh.rows, sh.can_run && !sh.run, sh.can_defer && !sh.defer};
    std::vector<Form> out{d};
    if (sh.can_group) out.push_back(Form{!d.group, d.rows, d.run_off, d.defer_off});
    if (sh.can_rows) out.push_back(Form{d.group, !d.rows, d.run_off, d.defer_off});
    if (sh.can_run) out.push_back(Form{d.group, d.rows, !d.run_off, d.defer_off});
    if (sh.can_defer) out.push_back(Form{d.group, d.rows, d.run_off, !d.defer_off});
    return out;
}

std::string form_code(const Shape &sh) {
    std::string c;
    c += sh.run ? 'R' : 'N';
    c += sh.group ? 'G' : 'W';
    c += sh.rows ? 'H' : 'h';
    c += sh.defer ? 'D' : 'd';
    return c;
}

std::string tune_key(const Prepared &P, size_t i, int wave) {
    const CNode &c = P.nodes[i];
    char buf[256];
    std::snprintf(buf, sizeof buf, "n%lld_m%lld_d%lld_w%d|kc%d|t%d_a%d_p%d_r%d|%s|wave%d|nb%d|chunk%d_p%d|",
                  (long long)P.n, (long long)P.g->nnz, (long long)P.g->max_degree, P.g->weighted ? 1 : 0, P.kc,
                  c.t, c.a, c.p, c.is_root ? 1 : 0, elem_name(P), wave, P.nb, P.g->chunk, P.g->panels);
    // the sub-template itself (nodes of one shape can be different trees);
    // its AHU form uses only parentheses, safe inside a JSON string
    return std::string(buf) + c.canon;
}

// The cache file: one flat JSON object {"key": "form code", ...}.
std::map<std::string, std::string> read_tune_cache(const char *path) {
    std::map<std::string, std::string> out;
    FILE *f = path ? std::fopen(path, "r") : nullptr;
    if (!f) return out;
    std::string text;
    char buf[4096];
    size_t r;
    while ((r = std::fread(buf, 1, sizeof buf, f)) > 0) text.append(buf, r);
    std::fclose(f);
    size_t pos = 0;
    while (true) {
        const size_t k0 = text.find('"', pos);
        if (k0 == std::string::npos) break;
        const size_t k1 = text.find('"', k0 + 1);
        const size_t v0 = k1 == std::string::npos ? k1 : text.find('"', k1 + 1);
        const size_t v1 = v0 == std::string::npos ? v0 : text.find('"', v0 + 1);
        if (v1 == std::string::npos) break;
        out[text.substr(k0 + 1, k1 - k0 - 1)] = text.substr(v0 + 1, v1 - v0 - 1);
        pos = v1 + 1;
    }
    return out;
}

void write_tune_cache(const char *path, const std::map<std::string, std::string> &m) {
    if (!path) return;
    const std::string tmp = std::string(path) + ".tmp";
    FILE *f = std::fopen(tmp.c_str(), "w");
    if (!f) return;
    std::fprintf(f, "{\n");
    size_t k = 0;
    for (const auto &kv : m)
        std::fprintf(f, "  \"%s\": \"%s\"%s\n", kv.first.c_str(), kv.second.c_str(), ++k < m.size() ? "," : "");
    std::fprintf(f, "}\n");
    std::fclose(f);
    std::rename(tmp.c_str(), path);
}

void set_form_code(Shape &sh, const std::string &code) {
    if (code.size() != 4) return;
    apply_form(sh, code[1] == 'G', code[2] == 'H', code[0] == 'N', code[3] == 'd');
}

sg2v_status tune_forms(sg2v_session *S, cudaStream_t stream) {
    Prepared &P = S->P;
    const size_t nn = P.nodes.size();
    const char *path = std::getenv("SG2V_TUNE_CACHE");
    std::map<std::string, std::string> cache = read_tune_cache(path);
    std::vector<std::vector<Form>> alts(nn);
    size_t most = 1;
    bool all_cached = true;
    for (size_t i = 0; i < nn; ++i) {
        alts[i] = form_alternatives(P.shape[i]);
        most = std::max(most, alts[i].size());
        if (!cache.count(tune_key(P, i, S->R.wave))) all_cached = false;
    }
    if (all_cached) {
        for (size_t i = 0; i < nn; ++i) set_form_code(P.shape[i], cache[tune_key(P, i, S->R.wave)]);
        return SG2V_OK;
    }
    std::vector<double> best(nn, -1.0);
    std::vector<std::string> best_code(nn);
    for (size_t k = 0; k < most; ++k) {
        for (size_t i = 0; i < nn; ++i) {
            const Form &f = alts[i][k < alts[i].size() ? k : 0];
            apply_form(P.shape[i], f.group, f.rows, f.run_off, f.defer_off);
        }
        sg2v_status st = session_enqueue(S, stream, false);  // warm-up
        if (st) return st;
        std::vector<double> ms(nn, 0.0);
        if ((st = session_enqueue(S, stream, false, false, &ms))) return st;
        for (size_t i = 0; i < nn; ++i) {
            if (k > 0 && k >= alts[i].size()) continue;
            if (best[i] < 0.0 || ms[i] < best[i]) {
                best[i] = ms[i];
                best_code[i] = form_code(P.shape[i]);
            }
        }
    }
    for (size_t i = 0; i < nn; ++i) {
        set_form_code(P.shape[i], best_code[i]);
        cache[tune_key(P, i, S->R.wave)] = best_code[i];
    }
    write_tune_cache(path, cache);
    return SG2V_OK;
}

sg2v_status graph_view(const sg2v_graph *g, int chunk, int panels, const sg2v_graph **out);

// Split schedule: the chunk size at which long rows are cut into tasks, and
// the number of column panels of the work list (1: none).  The session's
// whole step is timed (CUDA events, after a warm-up) on the work list of each
// candidate chunk size without panels, then on 2 and 4 panels at the best
// size, and the fastest is kept; SG2V_CHUNK fixes the chunk size and
// SG2V_PANELS the panels instead.  The choice is cached like the node forms,
// keyed by the graph statistics, colours, table type, colourings and the
// plans' sub-templates.
sg2v_status tune_split(sg2v_session *S, cudaStream_t stream) {
    const bool fix_chunk = std::getenv("SG2V_CHUNK") != nullptr;
    const bool fix_panels = std::getenv("SG2V_PANELS") != nullptr;
    if (fix_chunk && fix_panels) return SG2V_OK;
    Prepared &P = S->P;
    const sg2v_graph *base = S->base;
    const char *path = std::getenv("SG2V_TUNE_CACHE");
    std::map<std::string, std::string> cache = read_tune_cache(path);
    char buf[256];
    std::snprintf(buf, sizeof buf, "split|n%lld_m%lld_d%lld_w%d|kc%d|%s|nb%d|c%d_p%d|", (long long)P.n,
                  (long long)base->nnz, (long long)base->max_degree, base->weighted ? 1 : 0, P.kc, elem_name(P), P.nb,
                  fix_chunk ? base->chunk : 0, fix_panels ? base->panels : 0);
    std::string key(buf);
    for (const CNode &c : P.nodes)
        if (c.is_root) key += c.canon + ";";
    int best_c = base->chunk, best_p = base->panels;
    auto it = cache.find(key);
    if (it != cache.end() && std::sscanf(it->second.c_str(), "%d,%d", &best_c, &best_p) == 2) {
        // taken from the cache
    } else {
        cudaEvent_t a, b;
        SG2V_CUDA(cudaEventCreate(&a), "event");
        SG2V_CUDA(cudaEventCreate(&b), "event");
        float best_ms = 0.f;
        sg2v_status st = SG2V_OK;
        auto time_one = [&](int c, int pn) -> sg2v_status {
            const sg2v_graph *v = nullptr;
            sg2v_status s2 = graph_view(base, c, pn, &v);
            if (s2) return s2;
            P.g = v;
            if ((s2 = session_alloc_wave(S, P.auto_wave)))
                // a schedule whose scratch does not fit is not a candidate
                return s2 == SG2V_ERR_OUT_OF_MEMORY ? SG2V_OK : s2;
            if ((s2 = session_enqueue(S, stream, false))) return s2;  // warm-up
            SG2V_CUDA(cudaEventRecord(a, stream), "event");
            if ((s2 = session_enqueue(S, stream, false))) return s2;
            SG2V_CUDA(cudaEventRecord(b, stream), "event");
            SG2V_CUDA(cudaEventSynchronize(b), "event");
            float ms = 0.f;
            SG2V_CUDA(cudaEventElapsedTime(&ms, a, b), "event");
            if (best_ms == 0.f || ms < best_ms) {
                best_ms = ms;
                best_c = c;
                best_p = pn;
            }
            return SG2V_OK;
        };
        // chunk sizes below the largest degree (each splits some row) and the
        // first that splits none, without panels
        std::vector<int> cands;
        if (fix_chunk) {
            cands.push_back(base->chunk);
        } else {
            for (int c : {256, 512, 1024, 2048, 4096, 8192}) {
                cands.push_back(c);
                if (c >= base->max_degree) break;
            }
            if (std::find(cands.begin(), cands.end(), base->chunk) == cands.end()) cands.push_back(base->chunk);
        }
        const int p0 = fix_panels ? base->panels : 1;
        for (int c : cands)
            if ((st = time_one(c, p0))) break;
        if (!st && !fix_panels) {
            const int c = best_c;
            for (int pn : {2, 4})
                if ((st = time_one(c, pn))) break;
        }
        cudaEventDestroy(a);
        cudaEventDestroy(b);
        if (st) return st;
        cache[key] = std::to_string(best_c) + "," + std::to_string(best_p);
        write_tune_cache(path, cache);
    }
    const sg2v_graph *v = nullptr;
    sg2v_status st = graph_view(base, best_c, best_p, &v);
    if (st) return st;
    P.g = v;
    return session_alloc_wave(S, P.auto_wave);
}

int64_t count_launches(const Prepared &P, int wave) {
    const int64_t waves = (P.nb + wave - 1) / wave;
    int64_t per_wave = 1 + (int64_t)P.nodes.size() - (sort_hist_node(P) >= 0 ? 1 : 0);
    if (P.g->small_begin > 0 && P.g->small_begin < P.g->ntasks) per_wave += 1;  // two sort launches
    if (P.scaled)
        for (const CNode &c : P.nodes) per_wave += c.p != 1;
    const int whist = weighted_hist_node(P);  // one launch, whatever its shape
    for (size_t i = 0; i < P.shape.size(); ++i)
        if ((int)i != whist) per_wave += P.shape[i].defer + P.shape[i].group;
    return 1 + waves * per_wave + 2 * (int64_t)P.plans.size() + 1;
}

sg2v_status copy_out(double *dst, const double *src, size_t count, cudaStream_t stream) {
    if (!dst) return SG2V_OK;
    SG2V_CUDA(cudaMemcpyAsync(dst, src, count * sizeof(double), cudaMemcpyDefault, stream), "result copy");
    return SG2V_OK;
}

}  // namespace
}  // namespace sg2v

namespace sg2v {
namespace {

// The load-balanced work list of a graph for a chunk size: rows longer than
// `chunk` arcs are cut into chunk tasks sharing a split slot (the split
// schedule); sets the graph's task counts and boundaries, not its buffers.
// With panels > 1 (the column-panel form of the paper's CSC-Split, Alg. 6):
// the vertices that have arcs are cut into `panels` equal ranges; a row of
// more than kShortTaskArcs arcs (columns ascending) is also cut where its
// neighbours cross into the next range, and the tasks of each class (rows
// over kShortTaskArcs arcs, rows over kSortSmallArcs, the rest, then empty
// rows) run panel by panel (a shorter row goes with the panel of its first
// neighbour), so that the tasks in flight together gather from one range of
// the tables.  Every piece of a cut row shares its split slot and stays in
// the first class, which the one-task-per-warp kernels run.
void plan_worklist(sg2v_graph *g, const std::vector<int64_t> &rp, const std::vector<int32_t> &ci, int chunk,
                   int panels, std::vector<int4> *tasks_out, std::vector<int32_t> *hc_out) {
    const int64_t n = g->n;
    std::vector<int4> &tasks = *tasks_out;
    std::vector<int32_t> &hc = *hc_out;
    g->chunk = chunk;
    g->panels = std::max(1, panels);
    if (g->panels == 1 || ci.size() != (size_t)rp[(size_t)n]) {
        g->panels = 1;
        build_tasks(n, rp, chunk, &tasks, &hc);
    } else {
        // vertices with arcs come first when numbered by decreasing degree;
        // the ranges split them (a caller's order: all n vertices)
        int64_t live = n;
        while (live > 0 && rp[(size_t)live] == rp[(size_t)live - 1]) --live;
        const int64_t psize = std::max<int64_t>(1, (live + g->panels - 1) / g->panels);
        auto panel_of = [&](int64_t u) { return (int)std::min<int64_t>(g->panels - 1, u / psize); };
        std::vector<int32_t> order((size_t)n);
        for (int64_t i = 0; i < n; ++i) order[(size_t)i] = (int32_t)i;
        std::stable_sort(order.begin(), order.end(),
                         [&](int32_t x, int32_t y) { return rp[x + 1] - rp[x] > rp[y + 1] - rp[y]; });
        // [class][panel] task lists; class 0 long rows (and their pieces),
        // 1 rows of kSortSmallArcs+1 .. kShortTaskArcs arcs, 2 shorter, 3 empty
        std::vector<std::vector<std::vector<int4>>> bucket(4, std::vector<std::vector<int4>>((size_t)g->panels));
        for (int32_t v : order) {
            const int64_t e0 = rp[v], e1 = rp[v + 1], d = e1 - e0;
            if (d == 0) {
                bucket[3][0].push_back(make_int4(v, -1, (int)e0, (int)e1));
                continue;
            }
            if (d <= kShortTaskArcs) {
                // the panel of its first neighbour (the arcs come in column order)
                const int cls = d <= kSortSmallArcs ? 2 : 1;
                bucket[(size_t)cls][(size_t)panel_of(ci[(size_t)e0])].push_back(make_int4(v, -1, (int)e0, (int)e1));
                continue;
            }
            // pieces: panel boundaries, then chunks within a panel
            std::vector<int4> pieces;
            std::vector<int> ppanel;
            int64_t a = e0;
            while (a < e1) {
                const int pa = panel_of(ci[(size_t)a]);
                int64_t b = a + 1;
                while (b < e1 && panel_of(ci[(size_t)b]) == pa && b - a < chunk) ++b;
                pieces.push_back(make_int4(v, -1, (int)a, (int)b));
                ppanel.push_back(pa);
                a = b;
            }
            const int32_t slot = pieces.size() > 1 ? (int32_t)hc.size() : -1;
            if (slot >= 0) hc.push_back((int32_t)pieces.size());
            for (size_t k = 0; k < pieces.size(); ++k) {
                pieces[k].y = slot;
                bucket[0][(size_t)ppanel[k]].push_back(pieces[k]);
            }
        }
        tasks.clear();
        int64_t bounds[4];
        for (int cls = 0; cls < 4; ++cls) {
            for (const auto &bk : bucket[(size_t)cls]) tasks.insert(tasks.end(), bk.begin(), bk.end());
            bounds[cls] = (int64_t)tasks.size();
        }
        g->ntasks = (int64_t)tasks.size();
        g->nheavy = (int64_t)hc.size();
        g->short_begin = bounds[0];
        g->small_begin = bounds[1];
        g->live_tasks = bounds[2];
        g->live_rows = live;
        // forward counting skips the empty tasks only when their rows are the
        // last ones (vertices numbered by decreasing degree)
        bool tail = true;
        for (int64_t i = bounds[2]; i < g->ntasks; ++i)
            if (tasks[(size_t)i].x < live) tail = false;
        if (!tail) {
            g->live_tasks = g->ntasks;
            g->live_rows = n;
        }
        return;
    }
    g->ntasks = (int64_t)tasks.size();
    g->nheavy = (int64_t)hc.size();
    {
        int64_t nchunks = 0;
        for (int32_t c : hc) nchunks += c;
        g->short_begin = g->ntasks;
        for (int64_t i = nchunks; i < g->ntasks; ++i)
            if (tasks[(size_t)i].w - tasks[(size_t)i].z <= kShortTaskArcs) {
                g->short_begin = i;
                break;
            }
        g->small_begin = g->ntasks;
        for (int64_t i = g->short_begin; i < g->ntasks; ++i)
            if (tasks[(size_t)i].w - tasks[(size_t)i].z <= kSortSmallArcs) {
                g->small_begin = i;
                break;
            }
        // the work list's trailing empty tasks: skipped by forward counting
        // when their rows are exactly the last ones (each isolated vertex has
        // one empty task, every other row none)
        int64_t nempty = 0;
        while (nempty < g->ntasks && tasks[(size_t)(g->ntasks - 1 - nempty)].z == tasks[(size_t)(g->ntasks - 1 - nempty)].w)
            ++nempty;
        bool tail = true;
        for (int64_t i = g->ntasks - nempty; i < g->ntasks; ++i)
            if (tasks[(size_t)i].x < n - nempty) tail = false;
        g->live_tasks = tail ? g->ntasks - nempty : g->ntasks;
        g->live_rows = tail ? n - nempty : n;
    }
}

// A graph whose work list uses another chunk size or panel count (the graph
// itself when both are its own): built once per pair from the device CSR and
// kept with the graph, whose other arrays it shares.
sg2v_status graph_view(const sg2v_graph *g, int chunk, int panels, const sg2v_graph **out) {
    if ((chunk == g->chunk && panels == g->panels) || g->view) {
        *out = g;
        return SG2V_OK;
    }
    std::lock_guard<std::mutex> lock(g_mutex);
    for (const sg2v_graph *v : g->views)
        if (v->chunk == chunk && v->panels == panels) {
            *out = v;
            return SG2V_OK;
        }
    std::vector<int64_t> rp((size_t)g->n + 1);
    SG2V_CUDA(cudaMemcpy(rp.data(), g->row_ptr, rp.size() * sizeof(int64_t), cudaMemcpyDeviceToHost), "row pointers");
    std::vector<int32_t> ci;
    if (panels > 1) {
        ci.resize((size_t)g->nnz);
        SG2V_CUDA(cudaMemcpy(ci.data(), g->col_idx, ci.size() * sizeof(int32_t), cudaMemcpyDeviceToHost),
                  "column indices");
    }
    sg2v_graph *v = new (std::nothrow) sg2v_graph(*g);
    if (!v) return SG2V_ERR_OUT_OF_MEMORY;
    v->views.clear();
    v->view = true;
    v->tasks = nullptr;
    v->heavy_chunks = nullptr;
    v->rev = nullptr;
    std::vector<int4> tasks;
    std::vector<int32_t> hc;
    plan_worklist(v, rp, ci, chunk, panels, &tasks, &hc);
    cudaError_t e = cudaMalloc((void **)&v->tasks, std::max<size_t>(tasks.size() * sizeof(int4), 16));
    if (e == cudaSuccess && !tasks.empty())
        e = cudaMemcpy(v->tasks, tasks.data(), tasks.size() * sizeof(int4), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMalloc((void **)&v->heavy_chunks, std::max<size_t>(hc.size() * sizeof(int32_t), 16));
    if (e == cudaSuccess && !hc.empty())
        e = cudaMemcpy(v->heavy_chunks, hc.data(), hc.size() * sizeof(int32_t), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        free_graph(v);
        return cuda_fail(e, "work list upload");
    }
    const_cast<sg2v_graph *>(g)->views.push_back(v);
    *out = v;
    return SG2V_OK;
}

}  // namespace
}  // namespace sg2v

using namespace sg2v;

extern "C" {

sg2v_status sg2v_graph_create(int64_t n, int64_t nnz, const int64_t *row_ptr, const int32_t *col_idx,
                              const float *weights, uint32_t flags, sg2v_graph **out) {
    if (!out) {
        set_error("null output handle");
        return SG2V_ERR_INVALID_ARGUMENT;
    }
    *out = nullptr;
    if (n < 1 || n >= (int64_t(1) << 31) || nnz < 0 || nnz >= (int64_t(1) << 31) || !row_ptr ||
        (nnz > 0 && !col_idx) || (flags & ~(SG2V_GRAPH_SKIP_VALIDATION | SG2V_GRAPH_KEEP_ORDER))) {
        set_error("invalid graph size, pointer or flag");
        return SG2V_ERR_INVALID_ARGUMENT;
    }
    std::vector<int64_t> rp;
    std::vector<int32_t> ci;
    std::vector<float> w;
    sg2v_status st = host_copy(row_ptr, n + 1, &rp);
    if (st) return st;
    if ((st = host_copy(col_idx, nnz, &ci))) return st;
    if (weights && (st = host_copy(weights, nnz, &w))) return st;
    st = validate_csr(n, nnz, rp, ci, weights ? &w : nullptr, !(flags & SG2V_GRAPH_SKIP_VALIDATION));
    if (st) return st;
    std::vector<int32_t> iperm, arcmap;
    const bool relabel = !(flags & SG2V_GRAPH_KEEP_ORDER);
    if (relabel) relabel_by_degree(n, rp, ci, weights ? &w : nullptr, &iperm, &arcmap);

    int dev = 0;
    SG2V_CUDA(cudaGetDevice(&dev), "cudaGetDevice");
    sg2v_graph *g = new (std::nothrow) sg2v_graph();
    if (!g) return SG2V_ERR_OUT_OF_MEMORY;
    g->device = dev;
    g->n = n;
    g->nnz = nnz;
    g->weighted = weights != nullptr;
    for (int64_t i = 0; i < n; ++i) g->max_degree = std::max<int64_t>(g->max_degree, rp[i + 1] - rp[i]);
    // default chunk: 512 arcs up to an average degree of 64, else 1,024
    // (measured: rmat20_16m, rmat18_d16 and chunglu200k faster at 512,
    // rmat20_50m, average degree 95, at 1,024)
    g->chunk = env_int("SG2V_CHUNK", (double)nnz <= 64.0 * (double)n ? 512 : 1024);
    std::vector<int4> tasks;
    std::vector<int32_t> hc;
    plan_worklist(g, rp, ci, g->chunk, env_int("SG2V_PANELS", 1), &tasks, &hc);
    cudaError_t e = cudaSuccess;
    auto up = [&](void **dst, const void *src, size_t bytes) {
        if (e != cudaSuccess) return;
        e = cudaMalloc(dst, std::max<size_t>(bytes, 16));
        if (e == cudaSuccess && bytes) e = cudaMemcpy(*dst, src, bytes, cudaMemcpyHostToDevice);
    };
    up((void **)&g->row_ptr, rp.data(), rp.size() * sizeof(int64_t));
    up((void **)&g->col_idx, ci.data(), ci.size() * sizeof(int32_t));
    if (weights) up((void **)&g->weights, w.data(), w.size() * sizeof(float));
    up((void **)&g->tasks, tasks.data(), tasks.size() * sizeof(int4));
    up((void **)&g->heavy_chunks, hc.data(), hc.size() * sizeof(int32_t));
    if (relabel) {
        up((void **)&g->iperm, iperm.data(), iperm.size() * sizeof(int32_t));
        up((void **)&g->arcmap, arcmap.data(), arcmap.size() * sizeof(int32_t));
    }
    if (e != cudaSuccess) {
        free_graph(g);
        return cuda_fail(e, "graph upload");
    }
    *out = g;
    return SG2V_OK;
}

sg2v_status sg2v_graph_destroy(sg2v_graph *graph) {
    free_graph(graph);
    return SG2V_OK;
}

sg2v_status sg2v_graph_info(const sg2v_graph *g, int64_t *n, int64_t *nnz, int64_t *max_degree, int32_t *weighted) {
    if (!g) {
        set_error("null graph");
        return SG2V_ERR_INVALID_ARGUMENT;
    }
    if (n) *n = g->n;
    if (nnz) *nnz = g->nnz;
    if (max_degree) *max_degree = g->max_degree;
    if (weighted) *weighted = g->weighted ? 1 : 0;
    return SG2V_OK;
}

static sg2v_status count_batched_once(const sg2v_graph *g, const sg2v_plan *const *plans, int32_t num_plans,
                                      const int8_t *colours, int32_t B, sg2v_precision precision,
                                      double *per_vertex, double *totals, double *estimates, sg2v_stream stream_) {
    cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
    if (!colours) {
        set_error("null colours");
        return SG2V_ERR_INVALID_ARGUMENT;
    }
    Prepared P;
    sg2v_status st = prepare(g, plans, num_plans, B, precision, &P);
    if (st) return st;
    const int64_t n = P.n;
    const int nb = B;
    Workspace ws{stream, P.info.pool, {}};
    CallTimer timer(stream);
    // colours on the device
    const int8_t *d_col = colours;
    if (!is_device_pointer(colours)) {
        void *p;
        if ((st = ws.alloc(&p, (size_t)nb * n))) return st;
        SG2V_CUDA(cudaMemcpyAsync(p, colours, (size_t)nb * n, cudaMemcpyHostToDevice, stream), "colour upload");
        d_col = static_cast<const int8_t *>(p);
    }
    RunBuffers R;
    auto alloc = [&](size_t bytes, void **p) { return ws.alloc(p, bytes); };
    if ((st = alloc_run(P, P.auto_wave, alloc, &R))) return st;
    std::vector<double> ones_host;
    if (needs_ones(P)) {
        ones_host.assign((size_t)nb * n, 1.0);
        if ((st = ws.alloc((void **)&R.ones, ones_host.size() * sizeof(double)))) return st;
        SG2V_CUDA(cudaMemcpyAsync(R.ones, ones_host.data(), ones_host.size() * sizeof(double), cudaMemcpyHostToDevice,
                                  stream),
                  "fill");
    }
    // per-call tables from the stream-ordered pool, freed after their last consumer
    struct PoolTables : TableSource {
        Workspace &ws;
        std::vector<void *> &table;
        PoolTables(Workspace &w, std::vector<void *> &t) : ws(w), table(t) {}
        sg2v_status get(size_t i, size_t bytes, void **p) override { return ws.alloc(p, bytes); }
        void done(size_t i) override { ws.release(table[i]); }
    } src(ws, R.table);
    const bool pv_dev = per_vertex && is_device_pointer(per_vertex);
    double *pv_stage = nullptr;
    if (per_vertex && !pv_dev) {
        if ((st = ws.alloc((void **)&pv_stage, (size_t)num_plans * nb * n * sizeof(double)))) return st;
    }
    if ((st = enqueue(P, R, d_col, per_vertex ? (pv_dev ? per_vertex : pv_stage) : nullptr, src, stream, timer)))
        return st;
    std::vector<RootSum> sums((size_t)nb * num_plans);
    unsigned status[4] = {0, 0, 0, 0};
    SG2V_CUDA(cudaMemcpyAsync(sums.data(), R.sums, sums.size() * sizeof(RootSum), cudaMemcpyDeviceToHost, stream),
              "result copy");
    SG2V_CUDA(cudaMemcpyAsync(status, R.status, sizeof status, cudaMemcpyDeviceToHost, stream), "status copy");
    if (pv_stage)
        SG2V_CUDA(cudaMemcpyAsync(per_vertex, pv_stage, (size_t)num_plans * nb * n * sizeof(double),
                                  cudaMemcpyDeviceToHost, stream),
                  "per-vertex copy");
    SG2V_CUDA(cudaStreamSynchronize(stream), "stream synchronize");
    timer.collect();
    if (status[0] & 1u) {
        set_error("a colour is outside [0, num_colours)");
        return SG2V_ERR_COLOUR_OUT_OF_RANGE;
    }
    std::vector<double> tot(sums.size()), est(sums.size());
    bool nonfinite = (status[0] & 2u) != 0;  // an integer count wrapped past 2^64
    for (int pi = 0; pi < num_plans; ++pi) {
        for (int b = 0; b < nb; ++b) {
            const RootSum &r = sums[(size_t)pi * nb + b];
            long double t;
            if (r.flags & kFlagNonFinite) nonfinite = true;
            if (r.flags == 0) {
                unsigned __int128 x = ((unsigned __int128)r.hi << 64) | r.lo;
                tot[(size_t)pi * nb + b] = (double)x;  // correctly rounded conversion
                t = (long double)x;
            } else {
                tot[(size_t)pi * nb + b] = r.s + r.c;
                t = (long double)r.s + (long double)r.c;
            }
            est[(size_t)pi * nb + b] = (double)(t * plans[pi]->scale_ld);
        }
    }
    auto put = [&](double *dst, const std::vector<double> &src_) -> sg2v_status {
        if (!dst) return SG2V_OK;
        if (is_device_pointer(dst)) {
            SG2V_CUDA(cudaMemcpyAsync(dst, src_.data(), src_.size() * sizeof(double), cudaMemcpyHostToDevice, stream),
                      "result copy");
            SG2V_CUDA(cudaStreamSynchronize(stream), "stream synchronize");
        } else {
            std::memcpy(dst, src_.data(), src_.size() * sizeof(double));
        }
        return SG2V_OK;
    };
    if ((st = put(totals, tot))) return st;
    if ((st = put(estimates, est))) return st;
    if (nonfinite) {
        set_error("a count overflowed the table type");
        return SG2V_ERR_FP_OVERFLOW;
    }
    return SG2V_OK;
}

sg2v_status sg2v_count_batched(const sg2v_graph *g, const sg2v_plan *const *plans, int32_t num_plans,
                               const int8_t *colours, int32_t B, sg2v_precision precision, double *per_vertex,
                               double *totals, double *estimates, sg2v_stream stream) {
    sg2v_status st =
        count_batched_once(g, plans, num_plans, colours, B, precision, per_vertex, totals, estimates, stream);
    if (st == SG2V_ERR_FP_OVERFLOW && precision == SG2V_FP32)
        // FP32 tables ran out of exponent range: again with per-row exponents
        st = count_batched_once(g, plans, num_plans, colours, B, SG2V_FP32_SCALED, per_vertex, totals, estimates,
                                stream);
    return st;
}

sg2v_status sg2v_count(const sg2v_graph *graph, const sg2v_plan *plan, const int8_t *colours,
                       sg2v_precision precision, double *per_vertex, double *total, double *estimate,
                       sg2v_stream stream) {
    if (!plan) {
        set_error("null plan");
        return SG2V_ERR_INVALID_ARGUMENT;
    }
    const sg2v_plan *plans[1] = {plan};
    double t = 0.0, e = 0.0;
    sg2v_status st = sg2v_count_batched(graph, plans, 1, colours, 1, precision, per_vertex, &t, &e, stream);
    if (st == SG2V_OK || st == SG2V_ERR_FP_OVERFLOW) {
        if (total) *total = t;
        if (estimate) *estimate = e;
    }
    return st;
}

sg2v_status sg2v_session_create(const sg2v_graph *graph, const sg2v_plan *const *plans, int32_t num_plans,
                                int32_t B, sg2v_precision precision, uint32_t flags, sg2v_session **out) {
    if (!out || (flags & ~(SG2V_SESSION_PER_VERTEX | SG2V_SESSION_NO_GRAPH | SG2V_SESSION_AUTOTUNE))) {
        set_error("invalid argument");
        return SG2V_ERR_INVALID_ARGUMENT;
    }
    *out = nullptr;
    sg2v_session *S = new (std::nothrow) sg2v_session();
    if (!S) return SG2V_ERR_OUT_OF_MEMORY;
    S->flags = flags;
    S->hook = current_hook();
    S->base = graph;
    sg2v_status st = prepare(graph, plans, num_plans, B, precision, &S->P);
    if (st) {
        session_free(S);
        return st;
    }
    const Prepared &P = S->P;
    auto alloc = [&](size_t bytes, void **p) -> sg2v_status {
        sg2v_status s2 = session_malloc(S, bytes, p);
        if (s2) return s2;
        S->owned.push_back(*p);
        return SG2V_OK;
    };
    const size_t nseg = (size_t)num_plans * B;
    std::vector<double> scale(2 * num_plans);
    for (int pi = 0; pi < num_plans; ++pi) {
        scale[pi] = (double)plans[pi]->scale_ld;
        scale[num_plans + pi] = (double)(plans[pi]->scale_ld - (long double)scale[pi]);
    }
    cudaError_t e = cudaSuccess;
    if ((st = alloc((size_t)B * P.n, (void **)&S->colours)) || (st = alloc(nseg * sizeof(double), (void **)&S->totals)) ||
        (st = alloc(nseg * sizeof(double), (void **)&S->estimates)) ||
        (st = alloc(scale.size() * sizeof(double), (void **)&S->scale)) ||
        ((flags & SG2V_SESSION_PER_VERTEX) && (st = alloc(nseg * P.n * sizeof(double), (void **)&S->pv)))) {
        session_free(S);
        return st;
    }
    e = cudaMemcpy(S->scale, scale.data(), scale.size() * sizeof(double), cudaMemcpyHostToDevice);
    // wave-independent run buffers (the wave-dependent ones are replaced below)
    if (e == cudaSuccess && (st = alloc_run(P, 1, alloc, &S->R))) {
        session_free(S);
        return st;
    }
    if (e == cudaSuccess && needs_ones(P)) {
        std::vector<double> ones((size_t)B * P.n, 1.0);
        if ((st = alloc(ones.size() * sizeof(double), (void **)&S->R.ones))) {
            session_free(S);
            return st;
        }
        e = cudaMemcpy(S->R.ones, ones.data(), ones.size() * sizeof(double), cudaMemcpyHostToDevice);
    }
    if (e != cudaSuccess) {
        session_free(S);
        return cuda_fail(e, "session set-up");
    }
    if ((st = session_alloc_wave(S, P.auto_wave))) {
        session_free(S);
        return st;
    }
    S->tuned = !(flags & SG2V_SESSION_AUTOTUNE);
    S->launches_per_run = count_launches(P, S->R.wave);
    *out = S;
    return SG2V_OK;
}

sg2v_status sg2v_session_run(sg2v_session *S, const int8_t *colours, double *totals, double *estimates,
                             double *per_vertex, sg2v_stream stream_) {
    if (!S || !colours || (per_vertex && !S->pv)) {
        set_error("invalid argument (per_vertex needs SG2V_SESSION_PER_VERTEX)");
        return SG2V_ERR_INVALID_ARGUMENT;
    }
    cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
    const Prepared &P = S->P;
    sg2v_status st;
    SG2V_CUDA(cudaMemcpyAsync(S->colours, colours, (size_t)P.nb * P.n, cudaMemcpyDefault, stream), "colour copy");
    if (!S->tuned) {
        // the split schedule first, then the wave width, then each node's form
        if ((st = tune_split(S, stream))) return st;
        // time every candidate wave width on these colourings, keep the fastest
        std::vector<int> cands;
        for (int w = 1; w < P.nb; w *= 2) cands.push_back(w);
        cands.push_back(P.nb);
        if (std::find(cands.begin(), cands.end(), P.auto_wave) == cands.end()) cands.push_back(P.auto_wave);
        float best_ms = 0.f;
        int best = P.auto_wave;
        cudaEvent_t a, b;
        SG2V_CUDA(cudaEventCreate(&a), "event");
        SG2V_CUDA(cudaEventCreate(&b), "event");
        for (int w : cands) {
            if ((st = session_alloc_wave(S, w))) {
                if (st != SG2V_ERR_OUT_OF_MEMORY) return st;
                continue;  // a wave that does not fit is not a candidate
            }
            if ((st = session_enqueue(S, stream, false))) return st;  // warm-up
            SG2V_CUDA(cudaEventRecord(a, stream), "event");
            if ((st = session_enqueue(S, stream, false))) return st;
            SG2V_CUDA(cudaEventRecord(b, stream), "event");
            SG2V_CUDA(cudaEventSynchronize(b), "event");
            float ms = 0.f;
            SG2V_CUDA(cudaEventElapsedTime(&ms, a, b), "event");
            if (best_ms == 0.f || ms < best_ms) {
                best_ms = ms;
                best = w;
            }
        }
        cudaEventDestroy(a);
        cudaEventDestroy(b);
        if ((st = session_alloc_wave(S, best))) return st;
        if ((st = tune_forms(S, stream))) return st;
        S->tuned = true;
        S->launches_per_run = count_launches(P, best);
    }
    bool profiling;
    {
        std::lock_guard<std::mutex> lock(g_prof_mutex);
        profiling = g_prof_enabled;
    }
    if ((S->flags & SG2V_SESSION_NO_GRAPH) || profiling) {
        // direct launches (kernel timing records need them)
        if ((st = session_enqueue(S, stream, profiling))) return st;
    } else {
        if (!S->exec) {
            cudaGraph_t graph = nullptr;
            if (!S->capture) SG2V_CUDA(cudaStreamCreateWithFlags(&S->capture, cudaStreamNonBlocking), "stream");
            SG2V_CUDA(cudaStreamBeginCapture(S->capture, cudaStreamCaptureModeThreadLocal), "graph capture");
            st = session_enqueue(S, S->capture, false, true);
            cudaError_t e = cudaStreamEndCapture(S->capture, &graph);
            if (st) {
                if (graph) cudaGraphDestroy(graph);
                return st;
            }
            if (e != cudaSuccess) return cuda_fail(e, "graph capture");
            e = cudaGraphInstantiate(&S->exec, graph, 0);
            cudaGraphDestroy(graph);
            if (e != cudaSuccess) {
                S->exec = nullptr;
                return cuda_fail(e, "graph instantiate");
            }
        }
        SG2V_CUDA(cudaGraphLaunch(S->exec, stream), "graph launch");
        g_launches.fetch_add(S->launches_per_run);
    }
    const size_t nseg = P.plans.size() * (size_t)P.nb;
    if ((st = copy_out(totals, S->totals, nseg, stream))) return st;
    if ((st = copy_out(estimates, S->estimates, nseg, stream))) return st;
    if ((st = copy_out(per_vertex, S->pv, nseg * P.n, stream))) return st;
    return SG2V_OK;
}

sg2v_status sg2v_session_sync(sg2v_session *S, sg2v_stream stream_) {
    if (!S) {
        set_error("null session");
        return SG2V_ERR_INVALID_ARGUMENT;
    }
    cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
    unsigned status[4] = {0, 0, 0, 0};
    SG2V_CUDA(cudaMemcpyAsync(status, S->R.status, sizeof status, cudaMemcpyDeviceToHost, stream), "status copy");
    SG2V_CUDA(cudaStreamSynchronize(stream), "stream synchronize");
    if (status[0] & 1u) {
        set_error("a colour is outside [0, num_colours)");
        return SG2V_ERR_COLOUR_OUT_OF_RANGE;
    }
    if (status[0] & 2u) {
        set_error("a count overflowed the table type");
        return SG2V_ERR_FP_OVERFLOW;
    }
    return SG2V_OK;
}

sg2v_status sg2v_session_info(const sg2v_session *S, int32_t *wave, int32_t *graph) {
    if (!S) {
        set_error("null session");
        return SG2V_ERR_INVALID_ARGUMENT;
    }
    if (wave) *wave = S->R.wave;
    if (graph) *graph = S->exec != nullptr;
    return SG2V_OK;
}

sg2v_status sg2v_session_tuning(const sg2v_session *S, char *out, int64_t capacity, int64_t *length) {
    if (!S || (!out && capacity > 0)) {
        set_error("invalid argument");
        return SG2V_ERR_INVALID_ARGUMENT;
    }
    std::string j = "{\"wave\": " + std::to_string(S->R.wave) + ", \"chunk\": " + std::to_string(S->P.g->chunk) +
                    ", \"panels\": " + std::to_string(S->P.g->panels) +
                    ", \"tuned\": " + (S->tuned ? "true" : "false") + ", \"nodes\": [";
    for (size_t i = 0; i < S->P.nodes.size(); ++i) {
        const CNode &c = S->P.nodes[i];
        const Shape &sh = S->P.shape[i];
        const char *kernel = sh.rows ? "histogram rows" : (sh.run ? "run-scatter" : "per-colour accumulators");
        char buf[256];
        std::snprintf(buf, sizeof buf,
                      "%s{\"t\": %d, \"a\": %d, \"p\": %d, \"kernel\": \"%s\", \"lane_groups\": %s, "
                      "\"deferred_ema\": %s, \"form\": \"%s\"}",
                      i ? ", " : "", c.t, c.a, c.p, kernel, sh.group ? "true" : "false", sh.defer ? "true" : "false",
                      form_code(sh).c_str());
        j += buf;
    }
    j += "]}";
    if (length) *length = (int64_t)j.size();
    if (out && capacity > 0) {
        const size_t nb = std::min<size_t>((size_t)capacity - 1, j.size());
        std::memcpy(out, j.data(), nb);
        out[nb] = 0;
    }
    return SG2V_OK;
}

sg2v_status sg2v_session_destroy(sg2v_session *S) {
    session_free(S);
    return SG2V_OK;
}

sg2v_status sg2v_graph_set_weights(sg2v_graph *g, const float *weights, sg2v_stream stream_) {
    if (!g || !weights || !g->weighted) {
        set_error("graph must have been created with weights");
        return SG2V_ERR_INVALID_ARGUMENT;
    }
    cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
    if (!g->arcmap) {
        SG2V_CUDA(cudaMemcpyAsync(g->weights, weights, (size_t)g->nnz * sizeof(float), cudaMemcpyDefault, stream),
                  "weight copy");
        return SG2V_OK;
    }
    // the caller's arc order: staged, then gathered into the graph's order
    void *tmp = nullptr;
    SG2V_CUDA(cudaMallocAsync(&tmp, std::max<size_t>((size_t)g->nnz * sizeof(float), 16), stream), "allocation");
    cudaError_t e = cudaMemcpyAsync(tmp, weights, (size_t)g->nnz * sizeof(float), cudaMemcpyDefault, stream);
    if (e == cudaSuccess)
        e = launch_gather_f32(static_cast<const float *>(tmp), g->weights, g->arcmap, g->nnz, stream);
    cudaFreeAsync(tmp, stream);
    if (e != cudaSuccess) return cuda_fail(e, "weight copy");
    return SG2V_OK;
}

sg2v_status sg2v_count_backward(const sg2v_graph *g, const sg2v_plan *plan, const int8_t *colours,
                                sg2v_precision precision, const double *grad_per_vertex, double *grad_weights,
                                double *total, uint32_t flags, sg2v_stream stream_) {
    cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
    if (!g || !plan || !colours || !grad_weights ||
        (flags & ~(SG2V_BACKWARD_RECOMPUTE | SG2V_BACKWARD_STORE)) ||
        ((flags & SG2V_BACKWARD_RECOMPUTE) && (flags & SG2V_BACKWARD_STORE))) {
        set_error("invalid argument");
        return SG2V_ERR_INVALID_ARGUMENT;
    }
    if (precision == SG2V_FP32_SCALED || precision == SG2V_U64 || precision == SG2V_U128) {
        set_error("the backward pass keeps plain FP64 or FP32 tables");
        return SG2V_ERR_UNSUPPORTED;
    }
    const sg2v_plan *plans[1] = {plan};
    Prepared P;
    sg2v_status st = prepare(g, plans, 1, 1, precision, &P);
    if (st) return st;
    const int64_t n = P.n, nnz = g->nnz;
    const int kc = P.kc;
    const size_t esz = P.esz;
    const int vecn = P.vecn;
    sg2v_graph *gm = const_cast<sg2v_graph *>(g);
    if (!gm->rev) {
        // reverse arcs: arc (u, v) <-> arc (v, u); from host copies of the CSR
        std::vector<int64_t> rp((size_t)n + 1);
        std::vector<int32_t> ci((size_t)nnz), rv((size_t)nnz);
        SG2V_CUDA(cudaMemcpy(rp.data(), g->row_ptr, rp.size() * sizeof(int64_t), cudaMemcpyDeviceToHost), "copy");
        SG2V_CUDA(cudaMemcpy(ci.data(), g->col_idx, ci.size() * sizeof(int32_t), cudaMemcpyDeviceToHost), "copy");
        bool ok = true;
#pragma omp parallel for schedule(dynamic, 4096) reduction(&& : ok)
        for (int64_t u = 0; u < n; ++u)
            for (int64_t e = rp[u]; e < rp[u + 1]; ++e) {
                const int32_t v = ci[e];
                const int32_t *b0 = ci.data() + rp[v], *b1 = ci.data() + rp[v + 1];
                const int32_t *hit = std::lower_bound(b0, b1, (int32_t)u);
                if (hit == b1 || *hit != u) ok = false;
                else rv[e] = (int32_t)(hit - ci.data());
            }
        if (!ok) {
            set_error("CSR is not symmetric");
            return SG2V_ERR_GRAPH_NOT_SIMPLE;
        }
        SG2V_CUDA(cudaMalloc(&gm->rev, std::max<size_t>(rv.size() * sizeof(int32_t), 16)), "allocation");
        SG2V_CUDA(cudaMemcpy(gm->rev, rv.data(), rv.size() * sizeof(int32_t), cudaMemcpyHostToDevice), "copy");
    }
    Workspace ws{stream, P.info.pool, {}};
    CallTimer timer(stream);
    auto alloc = [&](size_t bytes, void **p) { return ws.alloc(p, bytes); };
    const int8_t *d_col = colours;
    if (!is_device_pointer(colours)) {
        void *p;
        if ((st = ws.alloc(&p, (size_t)n))) return st;
        SG2V_CUDA(cudaMemcpyAsync(p, colours, (size_t)n, cudaMemcpyHostToDevice, stream), "colour upload");
        d_col = static_cast<const int8_t *>(p);
    }
    if (g->iperm) {
        // the caller's colouring into the graph's vertex order
        void *p;
        if ((st = ws.alloc(&p, (size_t)n))) return st;
        SG2V_CUDA(launch_gather_i8(d_col, static_cast<int8_t *>(p), g->iperm, n, 1, stream), "colour permutation");
        d_col = static_cast<const int8_t *>(p);
    }
    double *gradw;
    if ((st = alloc((size_t)nnz * sizeof(double), (void **)&gradw))) return st;
    if (P.nodes.empty()) {
        // single-vertex template: the count does not depend on the weights
        SG2V_CUDA(cudaMemsetAsync(gradw, 0, (size_t)nnz * sizeof(double), stream), "memset");
        SG2V_CUDA(cudaMemcpyAsync(grad_weights, gradw, (size_t)nnz * sizeof(double), cudaMemcpyDefault, stream),
                  "copy");
        SG2V_CUDA(cudaStreamSynchronize(stream), "sync");
        if (total) *total = (double)n;
        return SG2V_OK;
    }
    // backward launch shapes of the transposed SpMM (gathers gradient rows of width C(kc-1, p))
    const size_t nn = P.nodes.size();
    std::vector<Shape> bshape(nn);
    // the backward tables of each node (cached per device and shape)
    std::vector<const BackwardTables *> btab(nn);
    std::vector<const uint32_t *> d_ybar(nn), d_mabar(nn), d_arc(nn);
    std::vector<const uint16_t *> d_bexp(nn);
    int64_t scratch_ld = P.scratch_ld;
    for (size_t i = 0; i < nn; ++i) {
        const CNode &c = P.nodes[i];
        Shape &sh = bshape[i];
        sh.wz = (int)binom(kc - 1, c.p);
        node_shape(P.vecn, sh.wz, &sh.grp, &sh.nv);
        if (sh.nv == 0) {
            set_error("gradient rows wider than this build's register tile");
            return SG2V_ERR_UNSUPPORTED;
        }
        sh.wz_pad = sh.grp * sh.nv * vecn;
        sh.ywords = ((int)binom(kc - 1, c.p - 1) + 3) / 4 * 4;
        sh.mwords = 0;
        if (sh.grp == kWideLanes) {
            sh.zwords = kc * sh.wz_pad;
            sh.threads = kWideThreads;
            sh.smem = (size_t)(sh.zwords + sh.ywords) * esz;
        } else {
            sh.zwords = (32 / sh.grp) * kc * sh.wz_pad;
            sh.threads = kNodeThreads;
            const size_t per_warp = (size_t)(sh.zwords + sh.ywords) * esz;
            while (sh.threads > 32 && (size_t)(sh.threads / 32) * per_warp > 200 * 1024) sh.threads /= 2;
            sh.smem = (size_t)(sh.threads / 32) * per_warp;
        }
        if (c.p >= 2) {
            sh.blocks_per_sm = node_blocks_per_sm(P.elem, false, sh.grp, sh.nv, g->weights != nullptr, sh.threads,
                                                  sh.smem);
            if (sh.blocks_per_sm < 1 || sh.smem > 227 * 1024) {
                set_error("transposed SpMM does not fit shared memory");
                return SG2V_ERR_UNSUPPORTED;
            }
            scratch_ld = std::max<int64_t>(scratch_ld, (int64_t)kc * sh.wz_pad);
        }
        const DeviceBackward *db = nullptr;
        if ((st = backward_tables(P.dev, kc, c.t, c.a, sh.wz_pad, &db))) return st;
        btab[i] = &db->host;
        d_ybar[i] = db->ybar;
        d_mabar[i] = db->mabar;
        d_arc[i] = db->arc;
        d_bexp[i] = db->expand;
    }
    // run buffers (one colouring), with split-row scratch wide enough for both directions
    Prepared Pw = P;
    Pw.scratch_ld = scratch_ld;
    RunBuffers R;
    if ((st = alloc_run(Pw, 1, alloc, &R))) return st;
    SG2V_CUDA(cudaMemsetAsync(R.status, 0, 16, stream), "memset");
    SG2V_CUDA(launch_check_colours(d_col, n, kc, R.status, stream), "colour check");
    SortHist no_hist{nullptr, 0, Elem::F32, nullptr, 0, nullptr};
    // the arc index of every sorted arc, for the per-arc gradient over sorted
    // arcs (SG2V_SDDMM_SORTED=0 keeps the per-row form)
    const char *sorted_env = std::getenv("SG2V_SDDMM_SORTED");
    const bool sorted_sddmm = !(sorted_env && std::atoi(sorted_env) == 0);
    int32_t *sperm = nullptr;
    if (sorted_sddmm) {
        if ((st = alloc((size_t)nnz * sizeof(int32_t), (void **)&sperm))) return st;
        no_hist.perm = sperm;
    }
    if (R.hcount) {
        // histogram nodes read each row's neighbour counts per colour from the
        // sort (unweighted graphs): split rows add theirs into a zeroed buffer
        SG2V_CUDA(cudaMemsetAsync(R.hcount, 0, (size_t)n * R.hld * sizeof(int32_t), stream), "memset");
        no_hist.hcount = R.hcount;
        no_hist.hld = R.hld;
    }
    SG2V_CUDA(launch_colour_sort(g->tasks, g->ntasks, g->small_begin, g->col_idx, g->weights, n, nnz, d_col, 1, kc,
                                 R.scol, R.sclr, R.sw, no_hist, P.info.sms, stream),
              "colour sort");
    std::vector<void *> yt(nn, nullptr), gt(nn, nullptr);
    std::vector<int64_t> ldy(nn, 0);
    for (size_t i = 0; i < nn; ++i) {
        ldy[i] = (binom(kc - 1, P.nodes[i].p) + vecn - 1) / vecn * vecn;
        if (!P.nodes[i].is_root) R.ld[i] = table_ld(P, P.nodes[i]);
    }
    // Stored form: the forward keeps every table, Y' and gradient table.
    // Recompute form (SG2V_BACKWARD_RECOMPUTE, or automatically when the
    // stored form would not fit 80% of free device memory): the forward
    // frees each table after its last consumer; the reverse walk brings back
    // the tables of the current node's children by replaying the forward of
    // their sub-templates (Alg. 5's bottom-up order, from the leaves), and
    // the node's Y' by replaying its gather, and frees all of it again.
    bool recompute = (flags & SG2V_BACKWARD_RECOMPUTE) != 0;
    if (!recompute && !(flags & SG2V_BACKWARD_STORE)) {
        double stored = 0.0;
        for (size_t i = 0; i < nn; ++i) {
            stored += (double)n * ldy[i] * esz;
            if (!P.nodes[i].is_root) stored += 2.0 * gather_table_bytes(n, 1, R.ld[i], esz);
        }
        size_t free_b = 0, total_b = 0;
        if (cudaMemGetInfo(&free_b, &total_b) == cudaSuccess) recompute = stored > 0.8 * (double)free_b;
        else cudaGetLastError();
    }
    // a node's children (distinct, not leaves)
    auto children = [&](size_t j) {
        std::vector<int> ch;
        const CNode &cj = P.nodes[j];
        if (cj.active != kLeaf) ch.push_back(cj.active);
        if (cj.passive != kLeaf && cj.passive != cj.active) ch.push_back(cj.passive);
        return ch;
    };
    // one forward node launch writing table j (Yout: also its Y')
    const int whist = weighted_hist_node(P);
    auto run_node = [&](size_t j, void *Yout) -> sg2v_status {
        if ((int)j == whist) {
            // weighted (2, 1, 1): table and Y' hold the same colour sums
            if (!R.table[j]) {
                sg2v_status s2 = alloc(gather_table_bytes(n, 1, R.ld[j], esz), &R.table[j]);
                if (s2) return s2;
                if ((s2 = zero_gather_row(R.table[j], n, 1, R.ld[j], esz, stream))) return s2;
            }
            if (g->nheavy) {  // chunks of split rows add into zeroed rows
                SG2V_CUDA(cudaMemsetAsync(R.table[j], 0, (size_t)n * R.ld[j] * esz, stream), "memset");
                if (Yout) SG2V_CUDA(cudaMemsetAsync(Yout, 0, (size_t)n * ldy[j] * esz, stream), "memset");
            }
            double b = (double)nnz * 5.0 + (double)n * (1.0 + (kc - 1) * (double)esz) + 16.0 * g->ntasks;
            if (Yout) b += (double)n * (kc - 1) * (double)esz;
            timer.begin(recompute ? "backward: recomputed forward node" : "backward: forward node", b);
            SG2V_CUDA(launch_weighted_hist(g->tasks, g->ntasks, g->small_begin, R.sclr, R.sw, nnz, d_col, n, 1, kc,
                                           R.table[j], R.ld[j], Yout, Yout ? ldy[j] : 0, P.elem, P.info.sms, stream),
                      "weighted histogram");
            timer.end();
            return SG2V_OK;
        }
        NodeArgs A = node_args(Pw, R, j, 0, 1, d_col);
        if (!P.nodes[j].is_root) {
            if (!R.table[j]) {
                sg2v_status s2 = alloc(gather_table_bytes(n, 1, R.ld[j], esz), &R.table[j]);
                if (s2) return s2;
                if ((s2 = zero_gather_row(R.table[j], n, 1, R.ld[j], esz, stream))) return s2;
            }
            A.Ms = R.table[j];
            A.ldt = R.ld[j];
        }
        if (Yout) {
            A.Yout = Yout;
            A.ldy = ldy[j];
        }
        if (g->nheavy) {
            SG2V_CUDA(cudaMemsetAsync(R.scratch, 0, R.scratch_bytes, stream), "memset");
            SG2V_CUDA(cudaMemsetAsync(R.counters, 0, R.counter_bytes, stream), "memset");
        }
        {
            const CNode &cj = P.nodes[j];
            const double rows = (double)n;
            double b = 8.0 * (n + 1) + (double)nnz * (5.0 + (g->weighted ? 4.0 : 0.0)) + rows;
            if (cj.p >= 2) b += rows * binom(kc - 1, cj.p - 1) * (double)esz;
            if (cj.a >= 2 && cj.active != cj.passive) b += rows * binom(kc - 1, cj.a - 1) * (double)esz;
            b += cj.is_root ? rows * (double)esz : rows * binom(kc - 1, cj.t - 1) * (double)esz;
            if (Yout) b += rows * binom(kc - 1, cj.p) * (double)esz;
            timer.begin(recompute ? "backward: recomputed forward node" : "backward: forward node", b);
        }
        SG2V_CUDA(launch_forward_node(P, j, A, stream), "node kernel launch");
        timer.end();
        return SG2V_OK;
    };
    auto drop_table = [&](int j) {
        if (j != kLeaf && R.table[(size_t)j]) {
            ws.release(R.table[(size_t)j]);
            R.table[(size_t)j] = nullptr;
        }
    };
    // recompute form: table j from its sub-template's leaves; tables of j's
    // children that `keep` does not hold are dropped again afterwards
    std::vector<char> keep(nn, 0);
    std::function<sg2v_status(int)> materialize = [&](int j) -> sg2v_status {
        if (j == kLeaf || R.table[(size_t)j]) return SG2V_OK;
        const std::vector<int> ch = children((size_t)j);
        for (int x : ch) {
            sg2v_status s2 = materialize(x);
            if (s2) return s2;
        }
        sg2v_status s2 = run_node((size_t)j, nullptr);
        if (s2) return s2;
        for (int x : ch)
            if (!keep[(size_t)x]) drop_table(x);
        return SG2V_OK;
    };
    if (!recompute) {
        // forward, keeping every table and every node's Y'
        for (size_t i = 0; i < nn; ++i) {
            if (!P.nodes[i].is_root) {
                if ((st = alloc((size_t)n * R.ld[i] * esz, &gt[i]))) return st;
                SG2V_CUDA(cudaMemsetAsync(gt[i], 0, (size_t)n * R.ld[i] * esz, stream), "memset");
            }
            if ((st = alloc((size_t)n * ldy[i] * esz, &yt[i]))) return st;
            if ((st = run_node(i, yt[i]))) return st;
        }
    } else {
        // forward for the total, each table dropped after its last consumer
        for (size_t i = 0; i < nn; ++i) {
            if ((st = run_node(i, nullptr))) return st;
            for (int x : children(i))
                if (P.nodes[(size_t)x].last_use == (int)i) drop_table(x);
        }
    }
    if (total) {
        timer.count_extra(2);
        SG2V_CUDA(launch_root_reduce(R.rootbuf[0], P.elem, n, n, 1, nullptr, nullptr, R.partials, R.chunks, R.sums, stream),
                  "root reduction");
    }
    // seed: gradient of the per-vertex counts
    double *seed;
    if ((st = alloc((size_t)n * sizeof(double), (void **)&seed))) return st;
    if (grad_per_vertex) {
        SG2V_CUDA(cudaMemcpyAsync(seed, grad_per_vertex, (size_t)n * sizeof(double), cudaMemcpyDefault, stream),
                  "seed copy");
        if (g->iperm) {
            // into the graph's vertex order
            double *seed2;
            if ((st = alloc((size_t)n * sizeof(double), (void **)&seed2))) return st;
            SG2V_CUDA(launch_gather_f64(seed, seed2, g->iperm, n, stream), "seed permutation");
            seed = seed2;
        }
    } else {
        std::vector<double> ones((size_t)n, 1.0);
        SG2V_CUDA(cudaMemcpyAsync(seed, ones.data(), ones.size() * sizeof(double), cudaMemcpyHostToDevice, stream),
                  "seed copy");
        SG2V_CUDA(cudaStreamSynchronize(stream), "sync");
    }
    double *part;
    if ((st = alloc((size_t)nnz * sizeof(double), (void **)&part))) return st;
    SG2V_CUDA(cudaMemsetAsync(part, 0, (size_t)nnz * sizeof(double), stream), "memset");
    // backward, parents before children
    for (size_t ii = nn; ii-- > 0;) {
        const CNode &c = P.nodes[ii];
        const int wy = (int)binom(kc - 1, c.p), wa = (int)binom(kc - 1, c.a - 1), ws_ = (int)binom(kc - 1, c.t - 1);
        if (recompute) {
            // the children's tables, this node's Y' (its table is rewritten
            // with the same values; the root's per-vertex values likewise),
            // and zeroed gradient tables for the children
            const std::vector<int> ch = children(ii);
            for (int x : ch) keep[(size_t)x] = 1;
            for (int x : ch)
                if ((st = materialize(x))) return st;
            if ((st = alloc((size_t)n * ldy[ii] * esz, &yt[ii]))) return st;
            if ((st = run_node(ii, yt[ii]))) return st;
            if (!c.is_root) drop_table((int)ii);
            for (int x : ch)
                if (!gt[(size_t)x]) {
                    if ((st = alloc((size_t)n * R.ld[(size_t)x] * esz, &gt[(size_t)x]))) return st;
                    SG2V_CUDA(cudaMemsetAsync(gt[(size_t)x], 0, (size_t)n * R.ld[(size_t)x] * esz, stream),
                              "memset");
                }
        }
        void *ybar;
        const int64_t ldyb = ldy[ii];
        if ((st = alloc(gather_table_bytes(n, 1, ldyb, esz), &ybar))) return st;
        if ((st = zero_gather_row(ybar, n, 1, ldyb, esz, stream))) return st;
        BwdEmaArgs E;
        std::memset(&E, 0, sizeof E);
        E.n = n;
        E.colours = d_col;
        E.kc = kc;
        E.a = c.a;
        E.ws = ws_;
        E.wa = c.a >= 2 ? wa : 0;
        E.wy = wy;
        E.G = c.is_root ? nullptr : gt[ii];
        E.ldg = R.ld[ii];
        E.seed = c.is_root ? seed : nullptr;
        if (c.a >= 2) {
            E.Ma = R.table[c.active];
            E.lda = R.ld[c.active];
            E.Gabar = gt[c.active];
            E.ldga = R.ld[c.active];
        }
        E.Y = yt[ii];
        E.ldy = ldy[ii];
        E.Ybar = ybar;
        E.ldyb = ldyb;
        E.ybar = d_ybar[ii];
        E.nybar = btab[ii]->nybar;
        E.mabar = d_mabar[ii];
        E.nmabar = btab[ii]->nmabar;
        {
            // algorithmic bytes: G (or the seed), M_a and Y' read, Ybar written,
            // the active child's gradient read and written
            const double rows = (double)n;
            double b = rows * ((c.is_root ? 8.0 : ws_ * (double)esz) + wy * (double)esz * 2.0);
            if (c.a >= 2) b += rows * wa * (double)esz * 3.0;
            timer.begin("backward: eMA", b);
        }
        SG2V_CUDA(launch_bwd_ema(E, P.fp64, P.info.sms, stream), "backward eMA");
        timer.end();
        if (c.p >= 2) {
            // gradient of the passive table: the transposed SpMM, colour-keyed like the forward
            const Shape &sh = bshape[ii];
            NodeArgs A = node_args(Pw, R, ii, 0, 1, d_col);
            A.hist = 0;
            A.Mp = ybar;
            A.ldp = ldyb;
            A.Wz = sh.wz;
            A.wz_pad = sh.wz_pad;
            A.zwords = sh.zwords;
            A.ywords = sh.ywords;
            A.mwords = 0;
            A.group_rows = 0;  // the transposed SpMM's shape is its own (one task per warp)
            A.defer = 0;
            A.npass = 1;
            A.zglobal = nullptr;
            A.p = btab[ii]->nterms;
            A.pstride = btab[ii]->nterms;
            A.wy = btab[ii]->wout;
            A.expand = d_bexp[ii];
            A.a_leaf = 1;
            A.Ma = nullptr;
            A.splits = nullptr;
            A.nsplit = 0;
            A.root = 0;
            A.root_out = nullptr;
            A.Ws = btab[ii]->wout;
            A.Ms = gt[c.passive];
            A.ldt = R.ld[c.passive];
            A.accumulate = 1;
            A.scratch_ld = scratch_ld;
            if (g->nheavy) {
                SG2V_CUDA(cudaMemsetAsync(R.scratch, 0, R.scratch_bytes, stream), "memset");
                SG2V_CUDA(cudaMemsetAsync(R.counters, 0, R.counter_bytes, stream), "memset");
            }
            // algorithmic bytes: the sorted arcs and row pointers, Ybar read once,
            // the passive child's gradient read and written
            timer.begin("backward: transposed SpMM",
                        (double)nnz * (5.0 + (g->weighted ? 4.0 : 0.0)) + 8.0 * (n + 1) +
                            (double)n * (wy + 2.0 * binom(kc - 1, c.p - 1)) * (double)esz);
            // on the run-scatter kernel where it has a variant for the row shape
            // (SG2V_BWD_RUN=0: per-colour accumulators and the expansion): each
            // colour run of neighbours' Ybar' rows goes through the transposed
            // run map straight into the gradient row, which it adds to
            const char *brun = std::getenv("SG2V_BWD_RUN");
            const bool run_ok = !(brun && std::atoi(brun) == 0) && !P.scaled && sh.grp != kWideLanes &&
                                (n + 1) * (ldyb / vecn) < (int64_t(1) << 28) &&
                                (sh.nv == 1 || (sh.nv == 2 && sh.grp == 32)) &&
                                (P.elem == Elem::F32 || (P.elem == Elem::F64 && !g->weights));
            int run_bps = 0;
            size_t run_smem = 0;
            const int rE = P.vecn;
            const int rybase = (btab[ii]->wout + rE - 1) / rE * rE;
            if (run_ok) {
                run_smem = (size_t)(kNodeThreads / 32) *
                           ((size_t)(32 / sh.grp) * (rybase + rE) * esz + (size_t)kRunCompactBytes);
                run_bps = node_run_blocks_per_sm(P.elem, sh.grp, sh.nv, g->weights != nullptr, 1, kNodeThreads,
                                                 run_smem);
            }
            if (run_bps >= 1) {
                const int wmap = sh.grp * sh.nv * rE;
                const uint16_t *rm = nullptr;
                if ((st = run_map(P.dev, kc, c.t, c.a, 3, wmap, rybase, &rm))) return st;
                NodeArgs Rn = A;
                Rn.runmap = rm;
                Rn.wmap = wmap;
                Rn.mzero = 0;
                Rn.ywords = rybase + rE;
                Rn.mwords = 0;
                Rn.half_arcs = 0;
                Rn.Yout = nullptr;
                SG2V_CUDA(launch_node_run(Rn, P.elem, sh.grp, sh.nv, 1, kNodeThreads, run_smem,
                                          P.info.sms * run_bps, stream),
                          "transposed SpMM launch");
            } else {
                SG2V_CUDA(launch_node(A, P.elem, sh.grp, sh.nv, sh.threads, sh.smem, P.info.sms * sh.blocks_per_sm,
                                      stream),
                          "transposed SpMM launch");
            }
            timer.end();
        }
        SddmmArgs D;
        std::memset(&D, 0, sizeof D);
        D.n = n;
        D.row_ptr = g->row_ptr;
        D.col_idx = g->col_idx;
        D.colours = d_col;
        D.kc = kc;
        D.hist = c.p == 1;
        D.Ybar = ybar;
        D.ldyb = ldyb;
        if (c.p >= 2) {
            D.Mp = R.table[c.passive];
            D.ldp = R.ld[c.passive];
        }
        D.wmp = (int)binom(kc - 1, c.p - 1);
        D.arc = d_arc[ii];
        D.narc = btab[ii]->narc;
        D.grad = part;
        // every form walks the forward work list (long rows in chunks)
        D.tasks = g->tasks;
        D.ntasks = g->ntasks;
        if (c.p >= 2) {
            // row-oriented form, gather shape of M_p' rows
            int lanes = 32, vecs = 1;
            node_shape(P.vecn, D.wmp, &lanes, &vecs);
            if (lanes != kWideLanes && vecs >= 1) {
                D.lanes = lanes;
                D.vecs = vecs;
                D.wz_pad = lanes * vecs * vecn;
                if (sorted_sddmm && sddmm_sorted_available(P.fp64, lanes, vecs)) {
                    // over the colour-sorted arcs: v's Ybar' row staged with a zero slot
                    const int ysink = (int)((wy + vecn - 1) / vecn * vecn);
                    const uint16_t *rm = nullptr;
                    if ((st = run_map(P.dev, kc, c.t, c.a, 0, lanes * vecs * vecn, ysink, &rm))) return st;
                    D.scol = R.scol;
                    D.sclr = R.sclr;
                    D.perm = sperm;
                    D.runmap = rm;
                    D.wmap = lanes * vecs * vecn;
                    D.ysink = ysink;
                    D.ywords = ysink + vecn;
                }
            }
        }
        // algorithmic bytes: the CSR, the colouring, Ybar and M_p read once,
        // the per-arc partial gradient read and written
        timer.begin("backward: SDDMM", (double)nnz * (4.0 + 16.0) + 8.0 * (n + 1) + (double)n +
                                           (double)n * (wy + (c.p >= 2 ? binom(kc - 1, c.p - 1) : 0)) * (double)esz);
        SG2V_CUDA(launch_sddmm(D, P.fp64, P.info.sms, stream), "SDDMM");
        timer.end();
        ws.release(ybar);
        if (recompute) {
            // this node is done: its Y', its gradient table and its children's
            // tables go (a table another parent reads is brought back there)
            ws.release(yt[ii]);
            yt[ii] = nullptr;
            if (gt[ii]) ws.release(gt[ii]);
            gt[ii] = nullptr;
            for (int x : children(ii)) {
                keep[(size_t)x] = 0;
                drop_table(x);
            }
        }
    }
    timer.count_extra(1);
    SG2V_CUDA(launch_symmetrize(part, g->rev, g->arcmap, nnz, gradw, stream), "symmetrize");
    SG2V_CUDA(cudaMemcpyAsync(grad_weights, gradw, (size_t)nnz * sizeof(double), cudaMemcpyDefault, stream),
              "gradient copy");
    RootSum sum;
    unsigned status[4] = {0, 0, 0, 0};
    if (total) SG2V_CUDA(cudaMemcpyAsync(&sum, R.sums, sizeof sum, cudaMemcpyDeviceToHost, stream), "copy");
    SG2V_CUDA(cudaMemcpyAsync(status, R.status, sizeof status, cudaMemcpyDeviceToHost, stream), "status copy");
    SG2V_CUDA(cudaStreamSynchronize(stream), "stream synchronize");
    timer.collect();
    if (status[0]) {
        set_error("a colour is outside [0, num_colours)");
        return SG2V_ERR_COLOUR_OUT_OF_RANGE;
    }
    if (total) {
        if (sum.flags == 0)
            *total = (double)(((unsigned __int128)sum.hi << 64) | sum.lo);
        else
            *total = sum.s + sum.c;
    }
    return SG2V_OK;
}

int64_t sg2v_last_call_peak_bytes(void) { return g_last_peak_bytes; }

sg2v_status sg2v_set_allocator(sg2v_alloc_fn alloc, sg2v_free_fn free_fn, void *user) {
    if ((alloc == nullptr) != (free_fn == nullptr)) {
        set_error("sg2v_set_allocator: give both functions or neither");
        return SG2V_ERR_INVALID_ARGUMENT;
    }
    std::lock_guard<std::mutex> lock(g_hook_mutex);
    g_hook.alloc = alloc;
    g_hook.free = free_fn;
    g_hook.user = alloc ? user : nullptr;
    return SG2V_OK;
}

const char *sg2v_status_string(sg2v_status s) {
    switch (s) {
        case SG2V_OK: return "ok";
        case SG2V_ERR_INVALID_ARGUMENT: return "invalid argument";
        case SG2V_ERR_NOT_A_TREE: return "template is not a tree";
        case SG2V_ERR_COLOUR_OUT_OF_RANGE: return "colour out of range";
        case SG2V_ERR_GRAPH_NOT_SIMPLE: return "graph is not simple and symmetric";
        case SG2V_ERR_OUT_OF_MEMORY: return "out of memory";
        case SG2V_ERR_FP_OVERFLOW: return "floating-point overflow";
        case SG2V_ERR_CUDA: return "CUDA error";
        case SG2V_ERR_TIMEOUT: return "device wait timed out";
        case SG2V_ERR_UNSUPPORTED: return "unsupported";
    }
    return "unknown status";
}

const char *sg2v_last_error(void) { return g_last_error.c_str(); }

sg2v_status sg2v_profile_enable(int32_t enable) {
    std::lock_guard<std::mutex> lock(g_prof_mutex);
    g_prof_enabled = enable != 0;
    return SG2V_OK;
}

sg2v_status sg2v_profile_reset(void) {
    std::lock_guard<std::mutex> lock(g_prof_mutex);
    g_prof.clear();
    g_launches.store(0);
    return SG2V_OK;
}

sg2v_status sg2v_profile_read(sg2v_kernel_record *out, int32_t capacity, int32_t *count) {
    if (!count || (capacity > 0 && !out)) {
        set_error("null argument");
        return SG2V_ERR_INVALID_ARGUMENT;
    }
    std::lock_guard<std::mutex> lock(g_prof_mutex);
    int32_t i = 0;
    for (auto &kv : g_prof) {
        if (i < capacity) {
            std::memset(&out[i], 0, sizeof out[i]);
            std::snprintf(out[i].name, sizeof out[i].name, "%s", kv.first.c_str());
            out[i].launches = kv.second.launches;
            out[i].total_ms = kv.second.total_ms;
            out[i].bytes_per_launch = kv.second.launches ? kv.second.bytes / (double)kv.second.launches : 0.0;
        }
        ++i;
    }
    *count = i;
    return SG2V_OK;
}

int64_t sg2v_launch_count(void) { return g_launches.load(); }

int32_t sg2v_version(void) { return 100; }

}  // extern "C"
