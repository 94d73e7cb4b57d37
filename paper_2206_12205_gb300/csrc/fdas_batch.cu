// Batched search: many series (dispersion-measure trials) of uneven length and zmax in one call.
//
// A batch holds one plan per series.  Series with the same (N, zmax, taps, segment length,
// precision) form a group that shares one template bank and twiddle tables (built once by the
// group's first plan).  fdas_batch_search runs every series through K1 -> K2/K3 -> K4 in one
// CUDA graph: the graph is captured on a library-owned stream the first time a set of buffers is
// seen and relaunched on the caller's stream afterwards, so a batch costs one launch on the host.
//
// Lanes: the series are spread over `lanes` concurrent branches of the graph (largest cost
// first, each to the least loaded lane), each branch with its own workspace slice and plane
// buffer sized for the largest series; inside a lane the series run back to back (stream order
// keeps a series' peak search ahead of the lane's next plane).  While one lane's plane kernel
// drains its last items or its small peak-search launches leave SMs idle, another lane's
// kernels fill them, and the launch gaps between kernels overlap.  Device memory is lanes x
// (workspace + plane) of the largest series, whatever the batch size.
//
// The autotuner (fdas_batch_autotune) times, for each FP32 group, the candidate segment lengths
// S in {1024, 2048, 4096, 8192} (S >= 2 taps) and templates per correlation CTA {1, 2, 4, 8, 16}
// on a zero spectrum and keeps the fastest (the tensor-core paths have no per-group launch
// choice: 4096-bin segments, one persistent CTA per SM); then it times the whole batch on a
// zero input at 1 .. 4 lanes and keeps the fastest.  Choices are cached in a small JSON file
// keyed by the device and the group's (or the batch's) shape.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <map>
#include <new>
#include <string>
#include <vector>

#include "fdas_internal.cuh"

using fdas::Plan;

struct fdas_plan_s : public fdas::Plan {};

struct fdas_batch_s {
    std::vector<fdas_config> cfg;          // per series (seg_len as tuned)
    std::vector<fdas_plan_s *> plan;       // per series
    std::vector<int> group;                // per series: index of its group
    std::vector<int> leader;               // per group: first series
    std::vector<std::string> key;          // per group: shape key
    std::vector<int64_t> sample_off;       // per series: element offset in the packed input
    std::vector<int64_t> peak_off;         // per series: record offset in the peak buffer
    int64_t total_samples = 0, total_peaks = 0, total_cells = 0;
    size_t ws_series = 0, plane_bytes = 0, ws_bytes = 0;
    bool templates_ready = false;
    int device = -1;
    cudaStream_t cap = nullptr;            // capture stream
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    const void *g_series = nullptr, *g_ws = nullptr, *g_peaks = nullptr, *g_npeaks = nullptr;
    int lanes = 1;                         // concurrent branches of the graph
    std::vector<int> lane_of;              // per series: its lane
    size_t lane_bytes = 0;                 // workspace slice of one lane (series scratch + plane)
    std::vector<cudaStream_t> lane_st;     // capture streams of the lanes
    std::vector<cudaEvent_t> lane_ev;      // fork (0) and the lanes' joins (1 ..)
    std::string last_error;
};

namespace {

constexpr size_t ALIGN = 256;
constexpr int BATCH_TUNE_LANES = 4;        // lane counts the autotuner times
size_t align_up(size_t x) { return (x + ALIGN - 1) & ~(ALIGN - 1); }
bool aligned(const void *ptr, uintptr_t a) { return (reinterpret_cast<uintptr_t>(ptr) & (a - 1)) == 0; }

fdas_status record(fdas_batch_s *b, cudaError_t e) {
    if (e == cudaSuccess) return FDAS_OK;
    if (b) b->last_error = std::string(cudaGetErrorName(e)) + ": " + cudaGetErrorString(e);
    (void)cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? FDAS_E_NOMEM : FDAS_E_CUDA;
}

fdas_status plan_one(const fdas_config &c, fdas_plan_s **out) {
    fdas_plan_t h = nullptr;
    size_t ws = 0;
    const fdas_status s = fdas_plan(&c, &h, &ws);
    *out = static_cast<fdas_plan_s *>(h);
    return s;
}

std::string group_key(const fdas_config &c) {
    char buf[160];
    std::snprintf(buf, sizeof buf, "p%d:n%lld:z%d:m%d:s%d:h%d", c.precision, (long long)c.n_samples, c.zmax, c.taps,
                  c.seg_len, c.harm_mode);
    return buf;
}

// Shape key of the autotune cache (segment length excluded: it is what gets chosen).
std::string tune_key(const fdas_config &c, int device) {
    cudaDeviceProp prop{};
    cudaGetDeviceProperties(&prop, device);
    char buf[200];
    std::snprintf(buf, sizeof buf, "sm%d%d_x%d:p%d:n%lld:z%d:m%d", prop.major, prop.minor, prop.multiProcessorCount,
                  c.precision, (long long)c.n_samples, c.zmax, c.taps);
    return buf;
}

// (Re)derive the per-series layout: groups, offsets, the shared workspace and plane buffer.
void layout(fdas_batch_s *b) {
    const int n = (int)b->plan.size();
    b->group.assign(n, -1);
    b->leader.clear();
    b->key.clear();
    b->sample_off.assign(n, 0);
    b->peak_off.assign(n, 0);
    std::map<std::string, int> gid;
    int64_t so = 0, po = 0, cells = 0;
    size_t ws = 0, pl = 0;
    for (int i = 0; i < n; i++) {
        const std::string k = group_key(b->cfg[i]);
        auto it = gid.find(k);
        if (it == gid.end()) {
            it = gid.emplace(k, (int)b->leader.size()).first;
            b->leader.push_back(i);
            b->key.push_back(k);
        }
        b->group[i] = it->second;
        b->sample_off[i] = so;
        b->peak_off[i] = po;
        so += b->cfg[i].n_samples;
        po += b->cfg[i].max_peaks;
        fdas_plan_info info{};
        fdas_plan_get_info(b->plan[i], &info);
        cells += info.cells;
        ws = std::max(ws, info.workspace_bytes);
        pl = std::max(pl, (size_t)info.plane_bytes);
    }
    b->total_samples = so;
    b->total_peaks = po;
    b->total_cells = cells;
    b->ws_series = align_up(ws);
    b->plane_bytes = align_up(pl);
    b->lane_bytes = b->ws_series + b->plane_bytes;
    b->ws_bytes = (size_t)b->lanes * b->lane_bytes;
    // lanes: largest cost (plane cells) first, each to the least loaded lane (lowest on ties)
    std::vector<int> idx(n);
    std::vector<int64_t> cost(n);
    for (int i = 0; i < n; i++) {
        idx[i] = i;
        cost[i] = (int64_t)(b->cfg[i].zmax + 1) * (b->cfg[i].n_samples / 2);
    }
    std::stable_sort(idx.begin(), idx.end(), [&](int a, int c) { return cost[a] > cost[c]; });
    std::vector<int64_t> load(b->lanes, 0);
    b->lane_of.assign(n, 0);
    for (int i : idx) {
        const int l = (int)(std::min_element(load.begin(), load.end()) - load.begin());
        b->lane_of[i] = l;
        load[l] += cost[i];
    }
}

void drop_graph(fdas_batch_s *b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
    b->g_series = b->g_ws = b->g_peaks = b->g_npeaks = nullptr;
}

// ---------------------------------------------------------------- autotune cache (JSON)
struct TuneChoice {
    int seg_len = 0, zb = 0, lanes = 0;    // lanes: batch entries only
    double ms = 0.0;
};

// One entry per line, as written by save_cache:
//   "  \"key\": {\"seg_len\": S, \"zb\": Z, \"lanes\": N, \"ms\": T},"
// (entries without the lanes field are read too)
std::map<std::string, TuneChoice> load_cache(const char *path) {
    std::map<std::string, TuneChoice> m;
    if (!path) return m;
    FILE *f = std::fopen(path, "r");
    if (!f) return m;
    char line[512];
    while (std::fgets(line, sizeof line, f)) {
        char key[256];
        TuneChoice c;
        if (std::sscanf(line, " \"%255[^\"]\": {\"seg_len\": %d, \"zb\": %d, \"lanes\": %d, \"ms\": %lf", key,
                        &c.seg_len, &c.zb, &c.lanes, &c.ms) == 5 ||
            std::sscanf(line, " \"%255[^\"]\": {\"seg_len\": %d, \"zb\": %d, \"ms\": %lf", key, &c.seg_len, &c.zb,
                        &c.ms) == 4)
            m[key] = c;
    }
    std::fclose(f);
    return m;
}

bool save_cache(const char *path, const std::map<std::string, TuneChoice> &m) {
    if (!path) return true;
    const std::string tmp = std::string(path) + ".tmp";
    FILE *f = std::fopen(tmp.c_str(), "w");
    if (!f) return false;
    std::fprintf(f, "{\n \"fdas_autotune\": 1,\n \"entries\": {\n");
    size_t k = 0;
    for (const auto &kv : m) {
        std::fprintf(f, "  \"%s\": {\"seg_len\": %d, \"zb\": %d, \"lanes\": %d, \"ms\": %.6f}%s\n",
                     kv.first.c_str(), kv.second.seg_len, kv.second.zb, kv.second.lanes, kv.second.ms,
                     ++k < m.size() ? "," : "");
    }
    std::fprintf(f, " }\n}\n");
    std::fclose(f);
    return std::rename(tmp.c_str(), path) == 0;
}

// Median-free timing: the best of `reps` event-timed fdas_plane calls (after one warm-up).
fdas_status time_plane(const fdas_config &c, int zb, cudaStream_t st, double *ms_out, std::string &err) {
    fdas_plan_s *p = nullptr;
    fdas_status s = plan_one(c, &p);
    if (s != FDAS_OK) return s;
    p->tune_zb = zb;
    s = fdas_make_templates(p, st);
    void *ws = nullptr, *xh = nullptr, *pl = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    fdas_plan_info info{};
    fdas_plan_get_info(p, &info);
    cudaError_t e = cudaSuccess;
    if (s == FDAS_OK) {
        e = cudaMalloc(&ws, info.workspace_bytes);
        if (e == cudaSuccess) e = cudaMalloc(&xh, sizeof(float2) * (size_t)info.nb);
        if (e == cudaSuccess) e = cudaMalloc(&pl, (size_t)info.plane_bytes);
        if (e == cudaSuccess) e = cudaMemsetAsync(xh, 0, sizeof(float2) * (size_t)info.nb, st);
        if (e == cudaSuccess) e = cudaEventCreate(&e0);
        if (e == cudaSuccess) e = cudaEventCreate(&e1);
        double best = 1e30;
        for (int r = 0; r < 4 && e == cudaSuccess && s == FDAS_OK; r++) {
            cudaEventRecord(e0, st);
            s = fdas_plane(p, static_cast<const float *>(xh), ws, pl, st);
            cudaEventRecord(e1, st);
            e = cudaEventSynchronize(e1);
            float ms = 0.f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
            if (r > 0) best = std::min(best, (double)ms);
        }
        *ms_out = best;
    }
    if (e != cudaSuccess) err = std::string(cudaGetErrorName(e)) + ": " + cudaGetErrorString(e);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(ws);
    cudaFree(xh);
    cudaFree(pl);
    fdas_destroy(p);
    if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? FDAS_E_NOMEM : FDAS_E_CUDA;
    return s;
}

// Cache key of a whole batch: the device and an FNV-1a digest of its series' shapes in order.
std::string batch_key(const fdas_batch_s *b, int device) {
    uint64_t h = 1469598103934665603ull;
    for (const fdas_config &c : b->cfg) {
        const std::string k = group_key(c);
        for (unsigned char ch : k) h = (h ^ ch) * 1099511628211ull;
        h = (h ^ 0xffu) * 1099511628211ull;
    }
    cudaDeviceProp prop{};
    cudaGetDeviceProperties(&prop, device);
    char buf[160];
    std::snprintf(buf, sizeof buf, "batch:sm%d%d_x%d:n%zu:h%016llx", prop.major, prop.minor, prop.multiProcessorCount,
                  b->plan.size(), (unsigned long long)h);
    return buf;
}

// The lanes' capture streams and the fork / join events (created on first use, kept until the
// batch is destroyed).
cudaError_t ensure_lanes(fdas_batch_s *b) {
    cudaError_t e = cudaSuccess;
    while ((int)b->lane_st.size() < b->lanes && e == cudaSuccess) {
        cudaStream_t st = nullptr;
        e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
        if (e == cudaSuccess) b->lane_st.push_back(st);
    }
    while ((int)b->lane_ev.size() < b->lanes + 1 && e == cudaSuccess) {
        cudaEvent_t ev = nullptr;
        e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
        if (e == cudaSuccess) b->lane_ev.push_back(ev);
    }
    return e;
}

// The best of two event-timed fdas_batch_search calls on a zero input at `lanes` lanes (after one
// call that captures the graph).  Buffers are the caller's (sized for the most lanes timed).
fdas_status time_batch(fdas_batch_s *b, int lanes, const float *series, void *ws, fdas_peak *peaks, int32_t *npeaks,
                       cudaStream_t st, double *ms_out) {
    fdas_status s = fdas_batch_set_lanes(b, lanes, nullptr);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    double best = 1e30;
    for (int r = 0; r < 3 && e == cudaSuccess && s == FDAS_OK; r++) {
        if (e == cudaSuccess) e = cudaEventRecord(e0, st);
        s = fdas_batch_search(b, series, ws, peaks, npeaks, st);
        if (e == cudaSuccess) e = cudaEventRecord(e1, st);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (r > 0) best = std::min(best, (double)ms);
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    *ms_out = best;
    if (s != FDAS_OK) return s;
    return record(b, e);
}

}  // namespace

extern "C" {

fdas_status fdas_batch_plan(const fdas_config *cfgs, int32_t n_series, fdas_batch_t *batch, size_t *workspace_bytes) {
    if (!cfgs || !batch || n_series <= 0) return FDAS_E_INVALID;
    *batch = nullptr;
    fdas_batch_s *b = new (std::nothrow) fdas_batch_s();
    if (!b) return FDAS_E_NOMEM;
    b->cfg.assign(cfgs, cfgs + n_series);
    for (int i = 0; i < n_series; i++) {
        fdas_plan_s *p = nullptr;
        const fdas_status s = plan_one(b->cfg[i], &p);
        if (s != FDAS_OK) {
            for (fdas_plan_s *q : b->plan) fdas_destroy(q);
            delete b;
            return s;
        }
        b->plan.push_back(p);
    }
    layout(b);
    *batch = b;
    if (workspace_bytes) *workspace_bytes = b->ws_bytes;
    return FDAS_OK;
}

fdas_status fdas_batch_autotune(fdas_batch_t b, const char *cache_path, void *stream) {
    if (!b) return FDAS_E_INVALID;
    if (b->templates_ready) return FDAS_E_STATE;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return record(b, e);
    std::map<std::string, TuneChoice> cache = load_cache(cache_path);
    bool changed = false;
    for (size_t g = 0; g < b->leader.size(); g++) {
        const fdas_config base = b->cfg[b->leader[g]];
        const std::string k = tune_key(base, dev);
        auto it = cache.find(k);
        TuneChoice choice;
        if (it != cache.end()) {
            choice = it->second;
        } else if (base.precision != FDAS_FP32) {
            choice.seg_len = base.seg_len;   // fixed 4096-bin tensor-core segments; nothing to choose
            choice.zb = 0;
            cache[k] = choice;
            changed = true;
        } else {
            double best = 1e30;
            for (int S = 1024; S <= 8192; S *= 2) {
                if (base.taps > S / 2) continue;
                for (int zb = 1; zb <= 16; zb *= 2) {
                    fdas_config c = base;
                    c.seg_len = S;
                    double ms = 0.0;
                    const fdas_status s = time_plane(c, zb, st, &ms, b->last_error);
                    if (s != FDAS_OK) return s;
                    if (ms < best) {
                        best = ms;
                        choice.seg_len = S;
                        choice.zb = zb;
                        choice.ms = ms;
                    }
                }
            }
            cache[k] = choice;
            changed = true;
        }
        // apply: re-plan the group's series with the chosen segment length and tile
        for (size_t i = 0; i < b->plan.size(); i++) {
            if (b->group[i] != (int)g) continue;
            fdas_config c = b->cfg[i];
            if (choice.seg_len > 0 && base.precision == FDAS_FP32) c.seg_len = choice.seg_len;
            fdas_plan_s *p = nullptr;
            const fdas_status s = plan_one(c, &p);
            if (s != FDAS_OK) return s;
            p->tune_zb = choice.zb;
            fdas_destroy(b->plan[i]);
            b->plan[i] = p;
            b->cfg[i] = c;
        }
    }
    layout(b);
    drop_graph(b);
    // lanes: the whole batch on a zero input (the plane and peak kernels' time hardly depends on
    // the data), 1 .. BATCH_TUNE_LANES lanes
    const std::string bk = batch_key(b, dev);
    auto bt = cache.find(bk);
    int lanes = 1;
    if (bt != cache.end() && bt->second.lanes >= 1 && bt->second.lanes <= FDAS_BATCH_MAX_LANES) {
        lanes = bt->second.lanes;
    } else {
        fdas_status s = fdas_batch_make_templates(b, stream);
        if (s != FDAS_OK) return s;
        const size_t ws_max = (size_t)BATCH_TUNE_LANES * b->lane_bytes;
        void *series = nullptr, *ws = nullptr, *peaks = nullptr, *npk = nullptr;
        e = cudaMalloc(&series, sizeof(float) * (size_t)b->total_samples);
        if (e == cudaSuccess) e = cudaMalloc(&ws, ws_max);
        if (e == cudaSuccess) e = cudaMalloc(&peaks, sizeof(fdas_peak) * (size_t)std::max<int64_t>(1, b->total_peaks));
        if (e == cudaSuccess) e = cudaMalloc(&npk, sizeof(int32_t) * b->plan.size());
        if (e == cudaSuccess) e = cudaMemsetAsync(series, 0, sizeof(float) * (size_t)b->total_samples, st);
        TuneChoice choice;
        double best = 1e30;
        for (int l = 1; l <= BATCH_TUNE_LANES && e == cudaSuccess && s == FDAS_OK; l++) {
            double ms = 0.0;
            s = time_batch(b, l, static_cast<const float *>(series), ws, static_cast<fdas_peak *>(peaks),
                           static_cast<int32_t *>(npk), st, &ms);
            if (s == FDAS_OK && ms < best) {
                best = ms;
                choice.lanes = l;
                choice.ms = ms;
            }
        }
        cudaFree(series);
        cudaFree(ws);
        cudaFree(peaks);
        cudaFree(npk);
        if (e != cudaSuccess) return record(b, e);
        if (s != FDAS_OK) return s;
        lanes = choice.lanes;
        cache[bk] = choice;
        changed = true;
    }
    fdas_batch_set_lanes(b, lanes, nullptr);
    if (changed && !save_cache(cache_path, cache)) {
        b->last_error = std::string("cannot write the autotune cache ") + cache_path;
        return FDAS_E_INVALID;
    }
    return FDAS_OK;
}

fdas_status fdas_batch_make_templates(fdas_batch_t b, void *stream) {
    if (!b) return FDAS_E_INVALID;
    if (b->templates_ready) return FDAS_OK;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaGetDevice(&b->device);
    if (e != cudaSuccess) return record(b, e);
    for (size_t g = 0; g < b->leader.size(); g++) {
        const fdas_status s = fdas_make_templates(b->plan[b->leader[g]], st);
        if (s != FDAS_OK) {
            b->last_error = fdas_last_error(b->plan[b->leader[g]]);
            return s;
        }
    }
    for (size_t i = 0; i < b->plan.size(); i++) {
        Plan *p = b->plan[i];
        const Plan *l = b->plan[b->leader[b->group[i]]];
        if (p == l) continue;
        p->device = l->device;
        p->d_tw = l->d_tw;
        p->d_twn_lo = l->d_twn_lo;
        p->d_twn_hi = l->d_twn_hi;
        p->d_G = l->d_G;
        p->d_Gbf = l->d_Gbf;
        p->d_tcF = l->d_tcF;
        p->d_tcTw = l->d_tcTw;
        p->d_Gh = l->d_Gh;
        p->d_tcFh = l->d_tcFh;
        p->d_dimg = l->d_dimg;
        p->d_dsig = l->d_dsig;
        p->d_k4order = l->d_k4order;
        p->k4order_n = l->k4order_n;
        p->d_k4order_a = l->d_k4order_a;
        p->k4order_a_n = l->k4order_a_n;
        p->borrowed = true;
        e = cudaMalloc((void **)&p->d_status, sizeof(int32_t));
        if (e == cudaSuccess) e = cudaMemsetAsync(p->d_status, 0, sizeof(int32_t), st);
        if (e != cudaSuccess) return record(b, e);
        p->templates_ready = true;
    }
    if (!b->cap) {
        e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
        if (e != cudaSuccess) return record(b, e);
    }
    e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return record(b, e);
    b->templates_ready = true;
    return FDAS_OK;
}

fdas_status fdas_batch_search(fdas_batch_t b, const float *d_series, void *d_workspace, fdas_peak *d_peaks,
                              int32_t *d_npeaks, void *stream) {
    if (!b || !d_series || !d_workspace || !d_npeaks || (!d_peaks && b->total_peaks > 0)) return FDAS_E_INVALID;
    if (!aligned(d_series, 8) || !aligned(d_workspace, 256) || !aligned(d_peaks, 4) || !aligned(d_npeaks, 4))
        return FDAS_E_INVALID;
    if (!b->templates_ready) return FDAS_E_STATE;
    // every series must start 8-byte aligned inside the packed input
    for (size_t i = 0; i < b->plan.size(); i++)
        if (!aligned(d_series + b->sample_off[i], 8)) return FDAS_E_INVALID;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (!(b->exec && b->g_series == d_series && b->g_ws == d_workspace && b->g_peaks == d_peaks &&
          b->g_npeaks == d_npeaks)) {
        drop_graph(b);
        cudaError_t e = ensure_lanes(b);
        if (e != cudaSuccess) return record(b, e);
        char *ws0 = static_cast<char *>(d_workspace);
        e = cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return record(b, e);
        // fork: every lane branches from the capture stream
        e = cudaEventRecord(b->lane_ev[0], b->cap);
        for (int l = 0; l < b->lanes && e == cudaSuccess; l++) e = cudaStreamWaitEvent(b->lane_st[l], b->lane_ev[0], 0);
        for (size_t i = 0; i < b->plan.size() && e == cudaSuccess; i++) {
            const Plan &p = *b->plan[i];
            const int lane = b->lane_of[i];
            cudaStream_t st_l = b->lane_st[lane];
            char *ws = ws0 + (size_t)lane * b->lane_bytes;
            void *plane = ws + b->ws_series;
            e = fdas::launch_spectrum(p, d_series + b->sample_off[i], ws, st_l);
            float2 *x = reinterpret_cast<float2 *>(ws + p.ws_x);
            const float *scale = reinterpret_cast<const float *>(ws + p.ws_scale + 8);
            if (e == cudaSuccess && p.cfg.norm_block) {
                e = fdas::launch_local_norm(p, x, x, st_l);
                scale = nullptr;
            }
            uint8_t *l1flag = fdas::level1_fusable(p) ? reinterpret_cast<uint8_t *>(ws + p.ws_l1flag) : nullptr;
            if (e == cudaSuccess) e = fdas::launch_plane_any(p, x, scale, ws, plane, st_l, l1flag);
            if (e == cudaSuccess)
                e = fdas::launch_peaks(p, plane, p.cfg.precision == FDAS_BF16 || p.cfg.precision == FDAS_BF16_DIRECT,
                                       ws, d_peaks + b->peak_off[i],
                                       d_npeaks + i, (uint32_t)i, st_l, l1flag, true);
        }
        // join: the capture stream waits for every lane
        for (int l = 0; l < b->lanes && e == cudaSuccess; l++) {
            e = cudaEventRecord(b->lane_ev[1 + l], b->lane_st[l]);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(b->cap, b->lane_ev[1 + l], 0);
        }
        cudaGraph_t g = nullptr;
        const cudaError_t e2 = cudaStreamEndCapture(b->cap, &g);
        if (e == cudaSuccess) e = e2;
        if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, g, 0);
        if (e != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            b->exec = nullptr;
            return record(b, e);
        }
        b->graph = g;
        b->g_series = d_series;
        b->g_ws = d_workspace;
        b->g_peaks = d_peaks;
        b->g_npeaks = d_npeaks;
    }
    return record(b, cudaGraphLaunch(b->exec, st));
}

fdas_status fdas_batch_set_lanes(fdas_batch_t b, int32_t lanes, size_t *workspace_bytes) {
    if (!b || lanes < 1 || lanes > FDAS_BATCH_MAX_LANES) return FDAS_E_INVALID;
    b->lanes = lanes;
    layout(b);
    drop_graph(b);
    if (workspace_bytes) *workspace_bytes = b->ws_bytes;
    return FDAS_OK;
}

fdas_status fdas_batch_get_info(fdas_batch_t b, int32_t *n_series, size_t *workspace_bytes, int64_t *total_samples,
                                int64_t *total_peaks, int64_t *total_cells) {
    if (!b) return FDAS_E_INVALID;
    if (n_series) *n_series = (int32_t)b->plan.size();
    if (workspace_bytes) *workspace_bytes = b->ws_bytes;
    if (total_samples) *total_samples = b->total_samples;
    if (total_peaks) *total_peaks = b->total_peaks;
    if (total_cells) *total_cells = b->total_cells;
    return FDAS_OK;
}

fdas_status fdas_batch_series_info(fdas_batch_t b, int32_t i, fdas_plan_info *info, fdas_config *cfg,
                                   int64_t *sample_offset, int64_t *peak_offset, int32_t *group) {
    if (!b || i < 0 || i >= (int32_t)b->plan.size()) return FDAS_E_INVALID;
    if (info) fdas_plan_get_info(b->plan[i], info);
    if (cfg) *cfg = b->cfg[i];
    if (sample_offset) *sample_offset = b->sample_off[i];
    if (peak_offset) *peak_offset = b->peak_off[i];
    if (group) *group = b->group[i];
    return FDAS_OK;
}

fdas_status fdas_batch_device_status(fdas_batch_t b, int32_t *bits, int clear) {
    if (!b || !bits) return FDAS_E_INVALID;
    int32_t acc = 0;
    for (fdas_plan_s *p : b->plan) {
        int32_t v = 0;
        const fdas_status s = fdas_device_status(p, &v, clear);
        if (s != FDAS_OK) return s;
        acc |= v;
    }
    *bits = acc;
    return FDAS_OK;
}

const char *fdas_batch_last_error(fdas_batch_t b) { return b ? b->last_error.c_str() : ""; }

void fdas_batch_destroy(fdas_batch_t b) {
    if (!b) return;
    if (b->device >= 0) cudaDeviceSynchronize();
    drop_graph(b);
    if (b->cap) cudaStreamDestroy(b->cap);
    for (cudaStream_t st : b->lane_st) cudaStreamDestroy(st);
    for (cudaEvent_t ev : b->lane_ev) cudaEventDestroy(ev);
    // followers first: they borrow their group leader's device memory
    for (size_t i = 0; i < b->plan.size(); i++)
        if (b->plan[i]->borrowed) fdas_destroy(b->plan[i]);
    for (size_t i = 0; i < b->plan.size(); i++)
        if (!b->plan[i]->borrowed) fdas_destroy(b->plan[i]);
    delete b;
}

}  // extern "C"
