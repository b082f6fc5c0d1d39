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
    const uint16_t *expand = nullptr;
    const uint32_t *splits = nullptr;
    int wy = 0, nsplit = 0;
};
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
    void *pe = nullptr, *ps = nullptr;
    const size_t be = tab.expand.size() * sizeof(uint16_t), bs = tab.splits.size() * sizeof(uint32_t);
    SG2V_CUDA(cudaMalloc(&pe, std::max<size_t>(be, 16)), "table upload");
    SG2V_CUDA(cudaMemcpy(pe, tab.expand.data(), be, cudaMemcpyHostToDevice), "table upload");
    if (bs) {
        SG2V_CUDA(cudaMalloc(&ps, bs), "table upload");
        SG2V_CUDA(cudaMemcpy(ps, tab.splits.data(), bs, cudaMemcpyHostToDevice), "table upload");
    }
    d.expand = static_cast<const uint16_t *>(pe);
    d.splits = static_cast<const uint32_t *>(ps);
    g_ctables[key] = d;
    *out = d;
    return SG2V_OK;
}

// ---- kernel timing records (measurement support)
struct ProfRecord {
    int64_t launches = 0;
    double total_ms = 0.0;
    double bytes = 0.0;
};
std::mutex g_prof_mutex;
bool g_prof_enabled = false;
std::map<std::string, ProfRecord> g_prof;
std::atomic<int64_t> g_launches{0};

// Event pairs of one call, folded into the records after its final sync.
struct CallTimer {
    bool on = false;
    struct Item {
        std::string name;
        double bytes;
        cudaEvent_t a, b;
    };
    std::vector<Item> items;
    cudaStream_t stream = nullptr;
    int open = -1;
    CallTimer(cudaStream_t s) : stream(s) {
        std::lock_guard<std::mutex> lock(g_prof_mutex);
        on = g_prof_enabled;
    }
    void begin(const std::string &name, double bytes) {
        g_launches.fetch_add(1);
        if (!on) return;
        Item it{name, bytes, nullptr, nullptr};
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
    void count_extra(int n) { g_launches.fetch_add(n); }
    // call after the stream has been synchronised
    void collect() {
        if (!on) return;
        std::lock_guard<std::mutex> lock(g_prof_mutex);
        for (auto &it : items) {
            float ms = 0.f;
            if (cudaEventElapsedTime(&ms, it.a, it.b) == cudaSuccess) {
                ProfRecord &r = g_prof[it.name];
                r.launches += 1;
                r.total_ms += ms;
                r.bytes = it.bytes;
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

// Allocations of one call, returned to the pool on every exit path.
struct Workspace {
    cudaStream_t stream;
    cudaMemPool_t pool;
    std::vector<void *> live;
    ~Workspace() {
        for (void *p : live) cudaFreeAsync(p, stream);
    }
    sg2v_status alloc(void **p, size_t bytes) {
        *p = nullptr;
        if (bytes == 0) bytes = 16;
        cudaError_t e = cudaMallocFromPoolAsync(p, bytes, pool, stream);
        if (e != cudaSuccess) return cuda_fail(e, "workspace allocation");
        live.push_back(*p);
        return SG2V_OK;
    }
    void release(void *p) {
        auto it = std::find(live.begin(), live.end(), p);
        if (it != live.end()) {
            cudaFreeAsync(p, stream);
            live.erase(it);
        }
    }
};

}  // namespace
}  // namespace sg2v

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
};

namespace sg2v {
namespace {

void free_graph(sg2v_graph *g) {
    if (!g) return;
    cudaFree(g->row_ptr);
    cudaFree(g->col_idx);
    cudaFree(g->weights);
    cudaFree(g->tasks);
    cudaFree(g->heavy_chunks);
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
    int bad = 0;  // 1: out of range, 2: not simple, 3: asymmetric, 4: bad weight
#pragma omp parallel for schedule(dynamic, 4096) reduction(max : bad)
    for (int64_t i = 0; i < n; ++i) {
        for (int64_t e = rp[i]; e < rp[i + 1]; ++e) {
            int32_t j = ci[e];
            if (j < 0 || j >= n) {
                bad = std::max(bad, 1);
                break;
            }
            if (!full) continue;
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
        case 1:
            set_error("col_idx entry out of range");
            return SG2V_ERR_INVALID_ARGUMENT;
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

struct CNode {
    int t, a, p;
    int active, passive;  // combined ids or kLeaf
    bool is_root;
    int last_use;
};

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
        (nnz > 0 && !col_idx) || (flags & ~SG2V_GRAPH_SKIP_VALIDATION)) {
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

    int dev = 0;
    SG2V_CUDA(cudaGetDevice(&dev), "cudaGetDevice");
    sg2v_graph *g = new (std::nothrow) sg2v_graph();
    if (!g) return SG2V_ERR_OUT_OF_MEMORY;
    g->device = dev;
    g->n = n;
    g->nnz = nnz;
    g->weighted = weights != nullptr;
    for (int64_t i = 0; i < n; ++i) g->max_degree = std::max<int64_t>(g->max_degree, rp[i + 1] - rp[i]);
    g->chunk = env_int("SG2V_CHUNK", 1024);
    std::vector<int4> tasks;
    std::vector<int32_t> hc;
    build_tasks(n, rp, g->chunk, &tasks, &hc);
    g->ntasks = (int64_t)tasks.size();
    g->nheavy = (int64_t)hc.size();
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

sg2v_status sg2v_count_batched(const sg2v_graph *g, const sg2v_plan *const *plans, int32_t num_plans,
                               const int8_t *colours, int32_t B, sg2v_precision precision, double *per_vertex,
                               double *totals, double *estimates, sg2v_stream stream_) {
    cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
    if (!g || !plans || num_plans < 1 || !colours || B < 1 || (precision != SG2V_FP64 && precision != SG2V_FP32)) {
        set_error("invalid argument");
        return SG2V_ERR_INVALID_ARGUMENT;
    }
    const int kc = plans[0] ? plans[0]->kc : 0;
    for (int i = 0; i < num_plans; ++i)
        if (!plans[i] || plans[i]->kc != kc) {
            set_error("plans must be non-null and share num_colours");
            return SG2V_ERR_INVALID_ARGUMENT;
        }
    int dev = 0;
    SG2V_CUDA(cudaGetDevice(&dev), "cudaGetDevice");
    if (dev != g->device) {
        set_error("graph lives on another device");
        return SG2V_ERR_INVALID_ARGUMENT;
    }
    DeviceInfo info;
    sg2v_status st = device_info(dev, &info);
    if (st) return st;
    const bool fp64 = precision == SG2V_FP64;
    const size_t esz = fp64 ? 8 : 4;
    const int vecn = fp64 ? 2 : 4;
    const int64_t n = g->n;
    const int nb = B;

    // ---- merged node list: sub-templates shared within and across plans
    std::vector<CNode> nodes;
    std::vector<int> plan_root(num_plans, -1);
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
                    pn.passive == kLeaf ? kLeaf : remap[pn.passive], pn.is_root, -1};
            nodes.push_back(c);
            remap[i] = (int)nodes.size() - 1;
            if (!pn.is_root) shared[pn.canon] = remap[i];
            if (pn.is_root) plan_root[pi] = remap[i];
        }
    }
    for (size_t i = 0; i < nodes.size(); ++i) {
        if (nodes[i].active != kLeaf) nodes[nodes[i].active].last_use = (int)i;
        if (nodes[i].passive != kLeaf) nodes[nodes[i].passive].last_use = (int)i;
    }
    // ---- per-node launch shape: gather width, Z layout, shared memory, block size
    struct Shape {
        int wz, grp, nv, wz_pad, zwords, ywords, mwords, threads;
        size_t smem;
    };
    std::vector<Shape> shape(nodes.size());
    int64_t scratch_ld = 1;
    for (size_t i = 0; i < nodes.size(); ++i) {
        const CNode &c = nodes[i];
        Shape &sh = shape[i];
        const bool hist = c.p == 1;
        sh.wz = hist ? 1 : (int)binom(kc - 1, c.p - 1);
        sh.grp = 32;
        sh.nv = 1;
        if (!hist) node_shape(fp64, sh.wz, &sh.grp, &sh.nv);
        if (sh.nv == 0) {
            set_error("passive table wider than this build's register tile (column tiling not built)");
            return SG2V_ERR_UNSUPPORTED;
        }
        sh.wz_pad = hist ? 1 : sh.grp * sh.nv * vecn;
        sh.zwords = hist ? (kc + 3) / 4 * 4 : (32 / sh.grp) * kc * sh.wz_pad;
        sh.ywords = ((int)binom(kc - 1, c.p) + 3) / 4 * 4;
        sh.mwords = c.a == 1 ? 0 : ((int)binom(kc - 1, c.a - 1) + 3) / 4 * 4;
        scratch_ld = std::max<int64_t>(scratch_ld, hist ? kc : (int64_t)kc * sh.wz_pad);
        sh.threads = kNodeThreads;
        const size_t per_warp = (size_t)(sh.zwords + sh.ywords + sh.mwords) * esz;
        while (sh.threads > 32 && (size_t)(sh.threads / 32) * per_warp > 200 * 1024) sh.threads /= 2;
        sh.smem = (size_t)(sh.threads / 32) * per_warp;
        if (sh.smem > 227 * 1024) {
            set_error("per-colour accumulators exceed shared memory (column tiling not built)");
            return SG2V_ERR_UNSUPPORTED;
        }
    }

    Workspace ws{stream, info.pool, {}};
    CallTimer timer(stream);
    // ---- colours on the device, range-checked there
    const int8_t *d_col = colours;
    if (!is_device_pointer(colours)) {
        void *p;
        if ((st = ws.alloc(&p, (size_t)nb * n))) return st;
        SG2V_CUDA(cudaMemcpyAsync(p, colours, (size_t)nb * n, cudaMemcpyHostToDevice, stream), "colour upload");
        d_col = static_cast<const int8_t *>(p);
    }
    unsigned *d_status;
    if ((st = ws.alloc((void **)&d_status, 16))) return st;
    SG2V_CUDA(cudaMemsetAsync(d_status, 0, 16, stream), "memset");
    timer.count_extra(1);
    SG2V_CUDA(launch_check_colours(d_col, (int64_t)nb * n, kc, d_status, stream), "colour check");

    // ---- every row's arcs sorted by neighbour colour, once per colouring
    int32_t *scol = nullptr;
    int8_t *sclr = nullptr;
    float *sw = nullptr;
    if ((st = ws.alloc((void **)&scol, (size_t)nb * g->nnz * sizeof(int32_t)))) return st;
    if ((st = ws.alloc((void **)&sclr, (size_t)nb * g->nnz))) return st;
    if (g->weighted && (st = ws.alloc((void **)&sw, (size_t)nb * g->nnz * sizeof(float)))) return st;
    timer.begin("colour_sort", (double)nb * (8.0 * (n + 1) + g->nnz * (4.0 + 4.0 + 1.0 + (g->weighted ? 8.0 : 0.0))));
    SG2V_CUDA(launch_colour_sort(g->tasks, g->ntasks, g->col_idx, g->weights, n, g->nnz, d_col, nb, kc, scol, sclr,
                                 sw, info.sms, stream),
              "colour sort");
    timer.end();

    // ---- scratch for split rows
    void *scratch = nullptr;
    unsigned *counters = nullptr;
    const size_t scratch_bytes = (size_t)(g->nheavy * nb * scratch_ld) * esz;
    const size_t counter_bytes = (size_t)(g->nheavy * nb) * sizeof(unsigned);
    if (g->nheavy) {
        if ((st = ws.alloc(&scratch, scratch_bytes))) return st;
        if ((st = ws.alloc((void **)&counters, counter_bytes))) return st;
    }

    // ---- the DP, children first
    std::vector<void *> table(nodes.size(), nullptr);
    std::vector<int64_t> ld(nodes.size(), 0);
    for (size_t i = 0; i < nodes.size(); ++i) {
        const CNode &c = nodes[i];
        NodeArgs A;
        std::memset(&A, 0, sizeof A);
        A.row_ptr = g->row_ptr;
        A.col_idx = g->col_idx;
        A.weights = g->weights;
        A.tasks = g->tasks;
        A.ntasks = g->ntasks;
        A.heavy_chunks = g->heavy_chunks;
        A.n = n;
        A.nb = nb;
        A.colours = d_col;
        A.kc = kc;
        A.nnz = g->nnz;
        A.scol = scol;
        A.sclr = sclr;
        A.sw = sw;
        const Shape &sh = shape[i];
        A.hist = c.p == 1;
        A.Wz = sh.wz;
        A.wz_pad = sh.wz_pad;
        A.zwords = sh.zwords;
        A.ywords = sh.ywords;
        A.mwords = sh.mwords;
        A.p = c.p;
        if (!A.hist) {
            A.Mp = table[c.passive];
            A.ldp = ld[c.passive];
        }
        A.a_leaf = c.a == 1;
        if (!A.a_leaf) {
            A.Ma = table[c.active];
            A.lda = ld[c.active];
            A.Wa = (int)binom(kc - 1, c.a - 1);
        }
        A.Ws = (int)binom(kc - 1, c.t - 1);
        DeviceTables tab;
        if ((st = device_tables(dev, kc, c.t, c.a, sh.wz_pad, &tab))) return st;
        A.expand = tab.expand;
        A.wy = tab.wy;
        A.splits = tab.splits;
        A.nsplit = tab.nsplit;
        A.root = c.is_root;
        if (c.is_root) {
            if ((st = ws.alloc(&table[i], (size_t)nb * n * esz))) return st;
            A.root_out = table[i];
        } else {
            ld[i] = (A.Ws + vecn - 1) / vecn * vecn;
            if ((st = ws.alloc(&table[i], (size_t)n * nb * ld[i] * esz))) return st;
            A.Ms = table[i];
            A.ldt = ld[i];
        }
        A.scratch = scratch;
        A.scratch_ld = scratch_ld;
        A.counters = counters;
        if (g->nheavy) {
            SG2V_CUDA(cudaMemsetAsync(scratch, 0, scratch_bytes, stream), "memset");
            SG2V_CUDA(cudaMemsetAsync(counters, 0, counter_bytes, stream), "memset");
        }
        const int bps = node_blocks_per_sm(fp64, A.hist, sh.grp, sh.nv, A.weights != nullptr, sh.threads, sh.smem);
        if (bps < 1) {
            set_error("node kernel cannot be resident with its shared memory");
            return SG2V_ERR_UNSUPPORTED;
        }
        {
            // algorithmic bytes: CSR once, each input table once, output once
            // (the sorted arc list: neighbour, its colour, weight)
            const double rows = (double)n * nb;
            double bytes = 8.0 * (n + 1) + (double)nb * g->nnz * (5.0 + (g->weighted ? 4.0 : 0.0));
            bytes += rows;  // colours
            if (!A.hist) bytes += rows * A.Wz * esz;
            if (!A.a_leaf && !(c.active == c.passive && !A.hist)) bytes += rows * binom(kc - 1, c.a - 1) * esz;
            bytes += c.is_root ? rows * esz : rows * A.Ws * esz;
            char name[64];
            std::snprintf(name, sizeof name, "node t=%d a=%d p=%d %s", c.t, c.a, c.p, fp64 ? "fp64" : "fp32");
            timer.begin(name, bytes);
        }
        SG2V_CUDA(launch_node(A, fp64, sh.grp, sh.nv, sh.threads, sh.smem, info.sms * bps, stream),
                  "node kernel launch");
        timer.end();
        if (c.active != kLeaf && nodes[c.active].last_use == (int)i) ws.release(table[c.active]);
        if (c.passive != kLeaf && nodes[c.passive].last_use == (int)i && c.passive != c.active)
            ws.release(table[c.passive]);
    }

    // ---- root reductions
    const bool pv_dev = per_vertex && is_device_pointer(per_vertex);
    double *pv_stage = nullptr;
    if (per_vertex && !pv_dev) {
        if ((st = ws.alloc((void **)&pv_stage, (size_t)num_plans * nb * n * sizeof(double)))) return st;
    }
    const int chunks = (int)std::max<int64_t>(1, std::min<int64_t>(256, (n + 65535) / 65536 * 4));
    RootSum *d_partials, *d_sums;
    if ((st = ws.alloc((void **)&d_partials, sizeof(RootSum) * (size_t)chunks * nb * num_plans))) return st;
    if ((st = ws.alloc((void **)&d_sums, sizeof(RootSum) * (size_t)nb * num_plans))) return st;
    double *ones = nullptr;
    for (int pi = 0; pi < num_plans; ++pi) {
        double *pv = per_vertex ? (pv_dev ? per_vertex : pv_stage) + (size_t)pi * nb * n : nullptr;
        const void *vals;
        bool vals_fp64 = fp64;
        if (plan_root[pi] >= 0) {
            vals = table[plan_root[pi]];
        } else {
            // single-vertex template: every vertex is one embedding
            if (!ones) {
                std::vector<double> h((size_t)nb * n, 1.0);
                if ((st = ws.alloc((void **)&ones, h.size() * sizeof(double)))) return st;
                SG2V_CUDA(cudaMemcpyAsync(ones, h.data(), h.size() * sizeof(double), cudaMemcpyHostToDevice, stream),
                          "fill");
                SG2V_CUDA(cudaStreamSynchronize(stream), "sync");
            }
            vals = ones;
            vals_fp64 = true;
        }
        timer.begin("root_reduce", (double)nb * n * ((vals_fp64 ? 8 : 4) + (pv ? 8 : 0)));
        timer.count_extra(1);
        SG2V_CUDA(launch_root_reduce(vals, vals_fp64, n, nb, pv, d_partials + (size_t)pi * nb * chunks, chunks,
                                     d_sums + (size_t)pi * nb, stream),
                  "root reduction");
        timer.end();
    }
    std::vector<RootSum> sums((size_t)nb * num_plans);
    unsigned status[4] = {0, 0, 0, 0};
    SG2V_CUDA(cudaMemcpyAsync(sums.data(), d_sums, sums.size() * sizeof(RootSum), cudaMemcpyDeviceToHost, stream),
              "result copy");
    SG2V_CUDA(cudaMemcpyAsync(status, d_status, sizeof status, cudaMemcpyDeviceToHost, stream), "status copy");
    if (pv_stage)
        SG2V_CUDA(cudaMemcpyAsync(per_vertex, pv_stage, (size_t)num_plans * nb * n * sizeof(double),
                                  cudaMemcpyDeviceToHost, stream),
                  "per-vertex copy");
    SG2V_CUDA(cudaStreamSynchronize(stream), "stream synchronize");
    timer.collect();
    if (status[0]) {
        set_error("a colour is outside [0, num_colours)");
        return SG2V_ERR_COLOUR_OUT_OF_RANGE;
    }
    std::vector<double> tot(sums.size()), est(sums.size());
    bool nonfinite = false;
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
    auto put = [&](double *dst, const std::vector<double> &src) -> sg2v_status {
        if (!dst) return SG2V_OK;
        if (is_device_pointer(dst)) {
            SG2V_CUDA(cudaMemcpyAsync(dst, src.data(), src.size() * sizeof(double), cudaMemcpyHostToDevice, stream),
                      "result copy");
            SG2V_CUDA(cudaStreamSynchronize(stream), "stream synchronize");
        } else {
            std::memcpy(dst, src.data(), src.size() * sizeof(double));
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
            out[i].bytes_per_launch = kv.second.bytes;
        }
        ++i;
    }
    *count = i;
    return SG2V_OK;
}

int64_t sg2v_launch_count(void) { return g_launches.load(); }

int32_t sg2v_version(void) { return 100; }

}  // extern "C"
