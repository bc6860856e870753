// device.cu -- C-ABI implementation of include/dpv.h: device state, the
// rank-commit state machine, scheduling (work list and fragment pool
// sizing) and kernel launches on the caller's stream.
//
// Collaborative semantics (arXiv 2407.00179 §3.2) are modelled on one
// process: dpvRenderFrame requires every logical rank to have committed its
// brick (the implicit barrier of anariRenderFrame), and the final frame is
// the one mapped "on rank 0" (§3.1.3).
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <map>
#include <string>
#include <vector>

#include "../../include/dpv.h"
#include "dpv_internal.cuh"
#include "launch.h"

using namespace dpv;

namespace {

thread_local std::string g_last_error;

dpv_status fail(dpv_status s, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return s;
}

struct HostBrick {
    bool committed = false;
    int lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
    int s_lo[3] = {0, 0, 0}, s_n[3] = {0, 0, 0};
    int dtype = 0;
    void* data = nullptr;       // device storage
    size_t bytes = 0;
    void* gather = nullptr;     // gather layout built from `data` (quad or cell)
    size_t gather_bytes = 0;
    int gather_kind = -1;       // GATHER_QUAD or GATHER_CELL
    bool gather_valid = false;
    float2* mm = nullptr;       // macro-cell value ranges (empty-space skipping)
    size_t mm_cells = 0;
    bool mm_valid = false;
};

const int kElemSize[4] = {4, 2, 2, 1};

}  // namespace

void dpv::set_last_error(const char* msg) { g_last_error = msg; }

const char* dpv::camera_problem(const dpv_camera& c) {
    float fx = c.center[0] - c.eye[0], fy = c.center[1] - c.eye[1], fz = c.center[2] - c.eye[2];
    float cx = fy * c.up[2] - fz * c.up[1], cy = fz * c.up[0] - fx * c.up[2], cz = fx * c.up[1] - fy * c.up[0];
    if (fx * fx + fy * fy + fz * fz == 0.0f) return "eye == center";
    if (cx * cx + cy * cy + cz * cz == 0.0f) return "up parallel to view";
    if (!(c.fovy_deg > 0.0f && c.fovy_deg < 180.0f)) return "fovy";
    return nullptr;
}

struct dpv_device_t {
    int nranks = 0;
    int cuda_device = 0;
    cudaStream_t stream = nullptr;
    bool poisoned = false;

    bool has_geom = false;
    int dims[3] = {0, 0, 0};
    float origin[3] = {0, 0, 0};
    float spacing = 1.0f;

    std::vector<HostBrick> bricks;
    float* d_scales = nullptr;          // per-rank scale (written by commit)
    unsigned int* d_tmp = nullptr;      // commit scratch (max |v|)
    BrickDev* d_bricks = nullptr;

    float4* d_tf = nullptr;
    int ntf = 0;
    float vmin = 0.f, vmax = 1.f;
    // host TF uploads: copied into one of two pinned staging slots, then
    // uploaded on the device stream (the caller's buffer is free at return
    // and the host does not wait for the device)
    float4* h_tf_stage[2] = {nullptr, nullptr};
    cudaEvent_t ev_tf_stage[2] = {nullptr, nullptr};
    int tf_stage_next = 0;
    bool has_light = false;
    float light_dir[3] = {0.f, 0.f, 1.f};   // unit, toward the light
    float light_step = 1.f;                 // h, voxels
    float light_ambient = 0.25f;            // k_a

    std::vector<CamIn> cams;
    CamIn* d_cam_in = nullptr;
    CamBasis* d_cams = nullptr;
    CamBasisDF* d_camd = nullptr;
    int cam_cap = 0;
    float4* d_rays = nullptr;           // per camera and pixel ray directions
    size_t rays_cap = 0;

    bool has_frame = false;
    dpv_frame_desc frame{};

    // schedule and buffers (rebuilt when dirty)
    bool dirty = true;
    FrameParams P{};
    int4* d_rects = nullptr;
    int* d_tile_count = nullptr;
    int* d_tile_first = nullptr;
    Item* d_items = nullptr;
    int items_cap = 0;
    int n_items = 0;
    float4* d_frag_rgba = nullptr;
    int* d_frag_key = nullptr;
    float4* d_frag_grad = nullptr;
    size_t frag_cap = 0;                // items the fragment pool holds
    float4* d_out_rgba = nullptr;
    float* d_out_depth = nullptr;
    unsigned char* d_order = nullptr;
    size_t out_cap = 0;                 // pixels the frame buffers hold
    size_t order_cap = 0;
    Counters* d_counters = nullptr;
    cudaEvent_t ev_done = nullptr;
    bool rendered = false;
    int gather = GATHER_QUAD;           // layout of the current frame

    // face adjoint buffer of the backward (float4 per cell face of every
    // brick) and each owner's neighbour list for the gather that follows
    float4* d_gface = nullptr;
    size_t gface_cap = 0;               // slots allocated
    size_t gface_slots = 0;             // slots the current bricks need
    size_t gface_tried = 0;             // slots asked for at the last allocation
    std::vector<size_t> gface_off_h;    // first slot of each brick (nranks + 1)
    unsigned char* d_empty = nullptr;   // macro-cell transparency of every brick
    size_t empty_cap = 0;
    int* d_tfz = nullptr;               // TF opaque-entry prefix counts (MAX_TF)
    int max_macro = 0;                  // most macro-cells of a brick
    int* d_nb_first = nullptr;          // nranks + 1
    int* d_nb = nullptr;                // nranks * nranks
    long long max_rows = 0;             // most owned (y, z) node rows of a brick

    // shadows by ray forwarding: per slot of the brick-major order its
    // record count and offset, the wave-fronts' first records, the records
    int* d_sh_counts = nullptr;
    long long* d_sh_offsets = nullptr;
    long long* d_sh_chunks = nullptr;
    long long* d_sh_total = nullptr;
    long long* d_rec_first = nullptr;   // nranks + 1
    size_t sh_slot_cap = 0;
    float4* d_recs = nullptr;
    long long rec_cap = 0;
    long long n_recs = 0;

    // persistent schedule (DPV_FRAME_PERSISTENT)
    int* d_sched = nullptr;
    int* d_hist = nullptr;              // nranks + 1 each
    int* d_offsets = nullptr;
    int* d_cursor = nullptr;
    unsigned long long* d_tmp64 = nullptr;
    unsigned int* d_work = nullptr;
    size_t sched_cap = 0;

    // asynchronous frame copies (dpvCopyFrameAsync): two staging slots,
    // each the frames of every camera, drained by a copy stream
    cudaStream_t copy_stream = nullptr;
    float4* d_stage_rgba[2] = {nullptr, nullptr};
    float* d_stage_depth[2] = {nullptr, nullptr};
    size_t stage_cap = 0;               // pixels per slot
    cudaEvent_t ev_staged[2] = {nullptr, nullptr};
    cudaEvent_t ev_drained[2] = {nullptr, nullptr};
    int stage_next = 0;

    // CUDA graph of the per-frame launches (DPV_FRAME_GRAPH)
    cudaStream_t cap_stream = nullptr;
    cudaGraphExec_t graph = nullptr;
    bool graph_failed = false;

    // profiling: event pairs around stages, resolved by dpvGetStats
    struct Timer {
        int stage;
        cudaEvent_t a, b;
    };
    bool profiling = false;
    std::vector<Timer> pending;
    std::vector<cudaEvent_t> event_pool;
    double stage_ms[DPV_NUM_STAGES] = {0};
    uint32_t stage_calls[DPV_NUM_STAGES] = {0};
    uint64_t launches = 0;
    uint64_t graph_launches = 0;

    // mapped fragment images (dpvMapFragments): per (camera, rank) a
    // device-owned block of width x height float4 RGBA then int32 keys
    struct FragMap {
        void* ptr;
        size_t bytes;
    };
    std::map<long long, FragMap> frag_maps;
};

namespace {

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        cudaGetDevice(&prev);
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur = -1;
        cudaGetDevice(&cur);
        if (prev >= 0 && cur != prev) cudaSetDevice(prev);
    }
};

dpv_status cuda_fail(dpv_device dev, cudaError_t e, const char* what) {
    if (dev) dev->poisoned = true;
    return fail(DPV_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define CK(call, what)                                      \
    do {                                                    \
        cudaError_t e_ = (call);                            \
        if (e_ != cudaSuccess) return cuda_fail(dev, e_, what); \
    } while (0)

dpv_status dev_alloc(dpv_device dev, void** p, size_t bytes, const char* what) {
    if (bytes == 0) bytes = 16;
    cudaError_t e = cudaMalloc(p, bytes);
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        *p = nullptr;
        return fail(DPV_ERR_OUT_OF_MEMORY, "%s: cannot allocate %zu bytes", what, bytes);
    }
    if (e != cudaSuccess) return cuda_fail(dev, e, what);
    return DPV_OK;
}

void dev_free(void* p) {
    if (p) cudaFree(p);
}

cudaEvent_t take_event(dpv_device dev) {
    if (!dev->event_pool.empty()) {
        cudaEvent_t e = dev->event_pool.back();
        dev->event_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return e;
}

// Record the start of a timed stage on the device stream (no-op when off).
cudaEvent_t stage_start(dpv_device dev) {
    if (!dev->profiling) return nullptr;
    cudaEvent_t e = take_event(dev);
    if (e) cudaEventRecord(e, dev->stream);
    return e;
}

void stage_stop(dpv_device dev, int stage, cudaEvent_t a) {
    if (!dev->profiling || !a) return;
    cudaEvent_t b = take_event(dev);
    if (!b) return;
    cudaEventRecord(b, dev->stream);
    dev->pending.push_back({stage, a, b});
}

// Wait for and accumulate all pending stage timers.
void resolve_timers(dpv_device dev) {
    for (auto& t : dev->pending) {
        float ms = 0.0f;
        if (cudaEventSynchronize(t.b) == cudaSuccess && cudaEventElapsedTime(&ms, t.a, t.b) == cudaSuccess) {
            dev->stage_ms[t.stage] += ms;
            dev->stage_calls[t.stage] += 1;
        }
        cudaGetLastError();
        dev->event_pool.push_back(t.a);
        dev->event_pool.push_back(t.b);
    }
    dev->pending.clear();
}

dpv_status check_dev(dpv_device dev) {
    if (!dev) return fail(DPV_ERR_INVALID_ARG, "null device");
    if (dev->poisoned) return fail(DPV_ERR_CUDA, "device is poisoned by an earlier CUDA error");
    return DPV_OK;
}

void free_schedule(dpv_device dev) {
    dev_free(dev->d_rects);
    dev_free(dev->d_tile_count);
    dev_free(dev->d_tile_first);
    dev_free(dev->d_items);
    dev->d_rects = nullptr;
    dev->d_tile_count = dev->d_tile_first = nullptr;
    dev->d_items = nullptr;
    dev->items_cap = 0;
}

void free_graph(dpv_device dev) {
    if (dev->graph) cudaGraphExecDestroy(dev->graph);
    dev->graph = nullptr;
    dev->graph_failed = false;
}

void free_shadow(dpv_device dev) {
    dev_free(dev->d_sh_counts);
    dev_free(dev->d_sh_offsets);
    dev_free(dev->d_sh_chunks);
    dev_free(dev->d_sh_total);
    dev_free(dev->d_rec_first);
    dev_free(dev->d_recs);
    dev->d_sh_counts = nullptr;
    dev->d_sh_offsets = nullptr;
    dev->d_sh_chunks = nullptr;
    dev->d_sh_total = nullptr;
    dev->d_rec_first = nullptr;
    dev->d_recs = nullptr;
    dev->sh_slot_cap = 0;
    dev->rec_cap = 0;
    dev->n_recs = 0;
}

void free_frags(dpv_device dev) {
    dev_free(dev->d_frag_rgba);
    dev_free(dev->d_frag_key);
    dev_free(dev->d_frag_grad);
    dev->d_frag_rgba = nullptr;
    dev->d_frag_key = nullptr;
    dev->d_frag_grad = nullptr;
    dev->frag_cap = 0;
}

// Owned ranges must tile [0, dims) exactly: every range non-empty and inside
// the volume, volumes summing to the total, and no two overlapping.
dpv_status check_partition(dpv_device dev) {
    long long total = 0;
    for (int k = 0; k < dev->nranks; ++k) {
        const HostBrick& b = dev->bricks[k];
        long long v = 1;
        for (int a = 0; a < 3; ++a) v *= (long long)(b.hi[a] - b.lo[a]);
        total += v;
        for (int m = k + 1; m < dev->nranks; ++m) {
            const HostBrick& c = dev->bricks[m];
            bool overlap = true;
            for (int a = 0; a < 3; ++a) overlap = overlap && b.lo[a] < c.hi[a] && c.lo[a] < b.hi[a];
            if (overlap) return fail(DPV_ERR_INVALID_ARG, "owned ranges of ranks %d and %d overlap", k, m);
        }
    }
    long long want = (long long)dev->dims[0] * dev->dims[1] * dev->dims[2];
    if (total != want)
        return fail(DPV_ERR_INVALID_ARG, "owned ranges cover %lld nodes, the volume has %lld", total, want);
    return DPV_OK;
}

// Whether the cell gather layout of every brick fits in half of the device
// memory that is free once the layouts held now are released.
bool cell_fits(dpv_device dev) {
    size_t need = 0, held = 0;
    for (const HostBrick& h : dev->bricks) {
        need += cell_bytes(h.dtype, h.s_n);
        if (h.gather) held += h.gather_bytes;
    }
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return need <= (free_b + held) / 2;
}

// Build FrameParams, upload the brick table, run the cull once to size the
// work list and fragment pool, and (re)allocate buffers.
dpv_status prepare(dpv_device dev) {
    const dpv_frame_desc& F = dev->frame;
    FrameParams& P = dev->P;
    P.W = F.width;
    P.H = F.height;
    P.tw = F.tile_w > 0 ? F.tile_w : 16;
    P.th = F.tile_h > 0 ? F.tile_h : 16;
    P.ntx = (P.W + P.tw - 1) / P.tw;
    P.nty = (P.H + P.th - 1) / P.th;
    P.ncam = (int)dev->cams.size();
    P.tp = P.tw * P.th;
    P.dt = F.step_voxels * dev->spacing;
    P.inv_dt = 1.0f / P.dt;
    P.sigma_max = F.sigma_max;
    P.ert = F.ert_threshold;
    P.ert_on = (F.ert_threshold > 0.0f && F.ert_threshold < 1.0f) ? 1 : 0;
    P.vmin = dev->vmin;
    P.vmax = dev->vmax;
    P.tf_scale = (float)(dev->ntf - 1) / (dev->vmax - dev->vmin);
    P.tf_bias = -P.vmin * P.tf_scale;
    P.sdt = P.sigma_max * P.dt;
    P.ntf = dev->ntf;
    for (int a = 0; a < 3; ++a) P.dims[a] = dev->dims[a];
    P.nbricks = dev->nranks;
    P.deep = (F.flags & DPV_FRAME_DEEP) ? DEEP_LAYERS : 1;
    P.order_stride = (F.flags & DPV_FRAME_ORDER) ? dev->nranks * P.deep : 0;
    P.items_cap = 0;
    // floats of shared memory per staged slab box; DPV_BOX_CAP overrides it
    // (tuning, and tests that force the unstaged fallback of large slabs)
    P.iso_on = (F.flags & DPV_FRAME_ISO) ? 1 : 0;
    P.ordered_on = (F.flags & DPV_FRAME_ORDERED) ? 1 : 0;
    P.skip_on = (F.flags & (DPV_FRAME_SKIP | DPV_FRAME_DEEP)) ? 1 : 0;   // deep fragments skip
    P.shadow_on = (F.flags & DPV_FRAME_SHADOW) ? 1 : 0;
    if (P.shadow_on && !dev->has_light) return fail(DPV_ERR_STATE, "DPV_FRAME_SHADOW needs dpvSetLight");
    for (int a = 0; a < 3; ++a) P.hl[a] = dev->light_step * dev->light_dir[a];
    P.shadow_dt = dev->light_step * dev->spacing;
    P.ambient = dev->light_ambient;
    P.iso = F.iso_value;
    P.box_cap = 6144;
    if (const char* env = getenv("DPV_BOX_CAP")) {
        int v = atoi(env);
        if (v >= 8 && v <= 40000) P.box_cap = v;
    }

    // brick table
    std::vector<BrickDev> table(dev->nranks);
    int dtype = dev->bricks[0].dtype;
    for (int k = 0; k < dev->nranks; ++k) {
        const HostBrick& h = dev->bricks[k];
        if (h.dtype != dtype) return fail(DPV_ERR_UNSUPPORTED, "all ranks must use the same storage dtype");
        BrickDev& b = table[k];
        b.data = h.data;
        for (int a = 0; a < 3; ++a) {
            b.s_lo[a] = h.s_lo[a];
            b.s_n[a] = h.s_n[a];
            float lo = (float)h.lo[a] - 0.5f, hi = (float)h.hi[a] - 0.5f;
            b.r0[a] = lo < 0.0f ? 0.0f : lo;
            b.r1[a] = hi > (float)(dev->dims[a] - 1) ? (float)(dev->dims[a] - 1) : hi;
            b.closed[a] = h.hi[a] >= dev->dims[a] ? 1 : 0;
        }
        b.sx = h.s_n[0];
        b.sxy = h.s_n[0] * h.s_n[1];
        b.scale_idx = k;
        b.pad = 0;
        b.gather = nullptr;
        b.qx = h.s_n[0] - 1;
        b.qxy = (h.s_n[0] - 1) * (h.s_n[1] - 1);
        for (int a = 0; a < 3; ++a) {
            b.o_lo[a] = h.lo[a];
            b.o_hi[a] = h.hi[a];
        }
    }
    // face adjoint buffer offsets, and per owner the bricks whose stored box
    // meets its owned box (itself first): the copies the gather sums
    {
        size_t off = 0;
        long long mo = 0;
        std::vector<int> first(dev->nranks + 1, 0), nb;
        dev->gface_off_h.assign(dev->nranks + 1, 0);
        for (int k = 0; k < dev->nranks; ++k) {
            const HostBrick& h = dev->bricks[k];
            table[k].gface_off = (long long)off;
            dev->gface_off_h[k] = off;
            off += face_slots(h.s_n);
            mo = std::max(mo, (long long)(h.hi[1] - h.lo[1]) * (h.hi[2] - h.lo[2]));
            first[k] = (int)nb.size();
            nb.push_back(k);
            for (int m = 0; m < dev->nranks; ++m) {
                if (m == k) continue;
                const HostBrick& c = dev->bricks[m];
                bool meet = true;
                for (int a = 0; a < 3; ++a) meet = meet && c.s_lo[a] < h.hi[a] && h.lo[a] < c.s_lo[a] + c.s_n[a];
                if (meet) nb.push_back(m);
            }
        }
        first[dev->nranks] = (int)nb.size();
        dev->gface_off_h[dev->nranks] = off;
        dev->gface_slots = off;
        dev->max_rows = mo;
        if (!dev->d_nb_first) {
            dpv_status s2 = dev_alloc(dev, (void**)&dev->d_nb_first, sizeof(int) * (MAX_RANKS + 1), "neighbour lists");
            if (s2) return s2;
            s2 = dev_alloc(dev, (void**)&dev->d_nb, sizeof(int) * MAX_RANKS * MAX_RANKS, "neighbour lists");
            if (s2) return s2;
        }
        CK(cudaMemcpyAsync(dev->d_nb_first, first.data(), sizeof(int) * first.size(), cudaMemcpyHostToDevice,
                           dev->stream), "upload neighbour lists");
        CK(cudaMemcpyAsync(dev->d_nb, nb.data(), sizeof(int) * nb.size(), cudaMemcpyHostToDevice, dev->stream),
           "upload neighbour lists");
        // the uploads read host vectors that end with this scope
        CK(cudaStreamSynchronize(dev->stream), "upload neighbour lists");
    }
    // gather layout (by flag, else cell where it fits, else quad): built
    // once per committed brick and layout
    const int kind = (F.flags & DPV_FRAME_LINEAR) ? GATHER_LINEAR
                     : (F.flags & DPV_FRAME_CELL) ? GATHER_CELL
                     : (F.flags & DPV_FRAME_QUAD) ? GATHER_QUAD
                     : cell_fits(dev)             ? GATHER_CELL
                                                  : GATHER_QUAD;
    if (kind != GATHER_LINEAR) {
        for (int k = 0; k < dev->nranks; ++k) {
            HostBrick& h = dev->bricks[k];
            size_t gb = kind == GATHER_CELL ? cell_bytes(h.dtype, h.s_n) : quad_bytes(h.dtype, h.s_n);
            if (h.gather && (h.gather_bytes != gb || h.gather_kind != kind)) {
                dev_free(h.gather);
                h.gather = nullptr;
                h.gather_valid = false;
            }
            if (!h.gather) {
                dpv_status s2 = dev_alloc(dev, &h.gather, gb, "gather layout");
                if (s2) return s2;
                h.gather_bytes = gb;
                h.gather_kind = kind;
                h.gather_valid = false;
            }
            if (!h.gather_valid) {
                if (kind == GATHER_CELL)
                    CK(launch_build_cell(h.dtype, h.data, h.s_n, h.gather, dev->stream), "build gather layout");
                else
                    CK(launch_build_quad(h.dtype, h.data, h.s_n, h.gather, dev->stream), "build gather layout");
                h.gather_valid = true;
            }
            table[k].gather = h.gather;
        }
    }
    dev->gather = kind;
    // the forward's quad gather uses pair-wide loads where a brick's layout
    // is far larger than L2 (its faces then come from DRAM): more than 6 L2.
    // Measured at 2048^3 (bricks of 514 nodes, 5 CTAs per SM): bf16 (layout
    // 8.2 L2) 192.8 ms with them, 199.6 without; fp8 (4.1 L2) 175.2 with,
    // 170.0 without
    P.quad_pair = 0;
    if (kind == GATHER_QUAD) {
        int l2 = 0;
        cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev->cuda_device);
        size_t biggest = 0;
        for (int k = 0; k < dev->nranks; ++k)
            biggest = std::max(biggest, quad_bytes(dev->bricks[k].dtype, dev->bricks[k].s_n));
        P.quad_pair = biggest > 6 * (size_t)l2 ? 1 : 0;
    }
    // empty-space skipping: per-brick macro-cell value ranges (once per
    // committed brick) and one transparency byte per macro-cell
    for (int k = 0; k < dev->nranks; ++k) {
        table[k].mm = nullptr;
        table[k].empty = nullptr;
        table[k].mx = table[k].mxy = table[k].mn = 0;
    }
    dev->max_macro = 0;
    if (P.skip_on) {
        size_t total = 0;
        for (int k = 0; k < dev->nranks; ++k) total += macro_cells(dev->bricks[k].s_n);
        if (total > dev->empty_cap) {
            dev_free(dev->d_empty);
            dev->d_empty = nullptr;
            dev->empty_cap = 0;
            dpv_status s2 = dev_alloc(dev, (void**)&dev->d_empty, total, "macro-cell transparency");
            if (s2) return s2;
            dev->empty_cap = total;
        }
        if (!dev->d_tfz) {
            dpv_status s2 = dev_alloc(dev, (void**)&dev->d_tfz, sizeof(int) * MAX_TF, "TF prefix");
            if (s2) return s2;
        }
        size_t off = 0;
        for (int k = 0; k < dev->nranks; ++k) {
            HostBrick& h = dev->bricks[k];
            const size_t mc = macro_cells(h.s_n);
            if (h.mm && h.mm_cells != mc) {
                dev_free(h.mm);
                h.mm = nullptr;
                h.mm_valid = false;
            }
            if (!h.mm) {
                dpv_status s2 = dev_alloc(dev, (void**)&h.mm, sizeof(float2) * mc, "macro-cell ranges");
                if (s2) return s2;
                h.mm_cells = mc;
                h.mm_valid = false;
            }
            if (!h.mm_valid) {
                CK(launch_build_minmax(h.dtype, h.data, h.s_n, h.mm, dev->stream), "macro-cell ranges");
                h.mm_valid = true;
            }
            table[k].mm = h.mm;
            table[k].empty = dev->d_empty + off;
            table[k].mx = ((h.s_n[0] - 2) >> MACRO_SHIFT) + 1;
            table[k].mxy = table[k].mx * (((h.s_n[1] - 2) >> MACRO_SHIFT) + 1);
            table[k].mn = (int)mc;
            dev->max_macro = std::max(dev->max_macro, (int)mc);
            off += mc;
        }
    }
    if (!dev->d_bricks) {
        dpv_status s = dev_alloc(dev, (void**)&dev->d_bricks, sizeof(BrickDev) * MAX_RANKS, "brick table");
        if (s) return s;
    }
    CK(cudaMemcpyAsync(dev->d_bricks, table.data(), sizeof(BrickDev) * dev->nranks, cudaMemcpyHostToDevice,
                       dev->stream), "upload brick table");

    // cameras
    if ((int)dev->cams.size() > dev->cam_cap) {
        dev_free(dev->d_cam_in);
        dev_free(dev->d_cams);
        dev_free(dev->d_camd);
        dev->d_cam_in = nullptr;
        dev->d_cams = nullptr;
        dev->d_camd = nullptr;
        dev->cam_cap = 0;
        dpv_status s = dev_alloc(dev, (void**)&dev->d_cam_in, sizeof(CamIn) * dev->cams.size(), "cameras");
        if (s) return s;
        s = dev_alloc(dev, (void**)&dev->d_cams, sizeof(CamBasis) * dev->cams.size(), "cameras");
        if (s) return s;
        s = dev_alloc(dev, (void**)&dev->d_camd, sizeof(CamBasisDF) * dev->cams.size(), "cameras");
        if (s) return s;
        dev->cam_cap = (int)dev->cams.size();
    }
    CK(cudaMemcpyAsync(dev->d_cam_in, dev->cams.data(), sizeof(CamIn) * dev->cams.size(), cudaMemcpyHostToDevice,
                       dev->stream), "upload cameras");

    // per-pixel ray directions
    size_t nrays = (size_t)P.ncam * P.W * P.H;
    if (nrays > dev->rays_cap) {
        dev_free(dev->d_rays);
        dev->d_rays = nullptr;
        dev->rays_cap = 0;
        dpv_status s2 = dev_alloc(dev, (void**)&dev->d_rays, RAY_VECS * sizeof(float4) * nrays, "rays");
        if (s2) return s2;
        dev->rays_cap = nrays;
    }
    P.rays = dev->d_rays;

    // schedule: count pass
    free_schedule(dev);
    size_t nct = (size_t)P.ncam * P.ntx * P.nty;
    dpv_status s;
    if ((s = dev_alloc(dev, (void**)&dev->d_rects, sizeof(int4) * (size_t)P.ncam * P.nbricks, "cull rects"))) return s;
    if ((s = dev_alloc(dev, (void**)&dev->d_tile_count, sizeof(int) * nct, "tile counts"))) return s;
    if ((s = dev_alloc(dev, (void**)&dev->d_tile_first, sizeof(int) * nct, "tile offsets"))) return s;
    if (!dev->d_counters) {
        if ((s = dev_alloc(dev, (void**)&dev->d_counters, sizeof(Counters), "counters"))) return s;
    }
    CK(cudaMemsetAsync(dev->d_counters, 0, sizeof(Counters), dev->stream), "reset counters");
    float3 og = make_float3(dev->origin[0], dev->origin[1], dev->origin[2]);
    CK(launch_cull(P, dev->d_cam_in, og, dev->spacing, dev->d_cams, dev->d_camd, dev->d_rays, dev->d_bricks, dev->d_rects,
                   dev->d_tile_count, dev->d_tile_first, nullptr, 0, dev->d_counters, false, dev->stream),
       "cull (sizing)");
    dev->launches += 4;
    Counters hc;
    CK(cudaMemcpyAsync(&hc, dev->d_counters, sizeof(Counters), cudaMemcpyDeviceToHost, dev->stream), "read counts");
    CK(cudaStreamSynchronize(dev->stream), "cull (sizing)");
    if (hc.n_items > (unsigned long long)0x7fffffff / (unsigned long long)P.tp)
        return fail(DPV_ERR_UNSUPPORTED, "work list too large (%llu items)", hc.n_items);
    dev->n_items = (int)hc.n_items;
    dev->items_cap = dev->n_items;
    P.items_cap = dev->items_cap;
    if ((s = dev_alloc(dev, (void**)&dev->d_items, sizeof(Item) * (size_t)std::max(1, dev->items_cap), "work list")))
        return s;
    // pull-order buffers of the persistent launches
    if ((size_t)std::max(1, dev->items_cap) > dev->sched_cap) {
        dev_free(dev->d_sched);
        dev->d_sched = nullptr;
        dev->sched_cap = 0;
        if ((s = dev_alloc(dev, (void**)&dev->d_sched, sizeof(int) * (size_t)std::max(1, dev->items_cap), "schedule")))
            return s;
        dev->sched_cap = (size_t)std::max(1, dev->items_cap);
    }
    if (!dev->d_hist) {
        if ((s = dev_alloc(dev, (void**)&dev->d_hist, sizeof(int) * (MAX_RANKS + 1) * 3 + 64, "schedule"))) return s;
        dev->d_offsets = dev->d_hist + (MAX_RANKS + 1);
        dev->d_cursor = dev->d_hist + 2 * (MAX_RANKS + 1);
        if ((s = dev_alloc(dev, (void**)&dev->d_tmp64, 64, "schedule"))) return s;
        dev->d_work = (unsigned int*)(dev->d_tmp64 + 1);
    }
    // an invalid item (all bits set) until the first fill writes the list
    CK(cudaMemsetAsync(dev->d_items, 0xFF, sizeof(Item) * (size_t)std::max(1, dev->items_cap), dev->stream),
       "clear work list");

    // fragment pool
    // (P.deep fragment layers per item)
    if ((size_t)dev->n_items * P.deep > dev->frag_cap) {
        free_frags(dev);
        size_t slots = (size_t)dev->n_items * P.deep * P.tp;
        if ((s = dev_alloc(dev, (void**)&dev->d_frag_rgba, sizeof(float4) * slots, "fragment pool"))) return s;
        if ((s = dev_alloc(dev, (void**)&dev->d_frag_key, sizeof(int) * slots, "fragment pool"))) return s;
        dev->frag_cap = (size_t)dev->n_items * P.deep;
    }
    // frame buffers
    size_t npix = (size_t)P.ncam * P.W * P.H;
    if (npix > dev->out_cap) {
        dev_free(dev->d_out_rgba);
        dev_free(dev->d_out_depth);
        dev->d_out_rgba = nullptr;
        dev->d_out_depth = nullptr;
        dev->out_cap = 0;
        if ((s = dev_alloc(dev, (void**)&dev->d_out_rgba, sizeof(float4) * npix, "frame"))) return s;
        if ((s = dev_alloc(dev, (void**)&dev->d_out_depth, sizeof(float) * npix, "frame"))) return s;
        dev->out_cap = npix;
    }
    size_t nord = npix * (size_t)P.order_stride;
    if (nord > dev->order_cap) {
        dev_free(dev->d_order);
        dev->d_order = nullptr;
        dev->order_cap = 0;
        if ((s = dev_alloc(dev, (void**)&dev->d_order, nord, "order image"))) return s;
        dev->order_cap = nord;
    }
    // shadow records: one per primary sample of every brick segment, sized
    // by one blocking pass over the filled work list
    if (P.shadow_on) {
        const size_t slots = (size_t)std::max(1, dev->n_items) * P.tp;
        if (slots > dev->sh_slot_cap) {
            free_shadow(dev);
            if ((s = dev_alloc(dev, (void**)&dev->d_sh_counts, sizeof(int) * slots, "shadow counts"))) return s;
            if ((s = dev_alloc(dev, (void**)&dev->d_sh_offsets, sizeof(long long) * slots, "shadow offsets")))
                return s;
            if ((s = dev_alloc(dev, (void**)&dev->d_sh_chunks,
                               sizeof(long long) * shadow_chunk_count(P, dev->n_items), "shadow offsets")))
                return s;
            if ((s = dev_alloc(dev, (void**)&dev->d_sh_total, sizeof(long long), "shadow offsets"))) return s;
            if ((s = dev_alloc(dev, (void**)&dev->d_rec_first, sizeof(long long) * (MAX_RANKS + 1), "wave-fronts")))
                return s;
            dev->sh_slot_cap = slots;
        }
        CK(launch_cull(P, dev->d_cam_in, og, dev->spacing, dev->d_cams, dev->d_camd, dev->d_rays, dev->d_bricks,
                       dev->d_rects, dev->d_tile_count, dev->d_tile_first, dev->d_items, dev->items_cap,
                       dev->d_counters, true, dev->stream),
           "cull (shadow sizing)");
        CK(launch_schedule(P, dev->d_items, dev->n_items, 1, dev->d_hist, dev->d_offsets, dev->d_cursor,
                           dev->d_tmp64, dev->d_sched, dev->stream),
           "schedule (shadow sizing)");
        CK(launch_shadow_offsets(P, dev->d_cams, dev->d_bricks, dev->d_items, dev->n_items, dev->d_sched,
                                 dev->d_sh_counts, dev->d_sh_offsets, dev->d_sh_chunks, dev->d_sh_total,
                                 dev->stream),
           "shadow sizing");
        long long total = 0;
        CK(cudaMemcpyAsync(&total, dev->d_sh_total, sizeof total, cudaMemcpyDeviceToHost, dev->stream),
           "shadow sizing");
        CK(cudaStreamSynchronize(dev->stream), "shadow sizing");
        dev->launches += 14;
        if (total > dev->rec_cap) {
            dev_free(dev->d_recs);
            dev->d_recs = nullptr;
            dev->rec_cap = 0;
            if ((s = dev_alloc(dev, (void**)&dev->d_recs, sizeof(float4) * (size_t)std::max(1LL, total),
                               "shadow rays")))
                return s;
            dev->rec_cap = total;
        }
        dev->n_recs = total;
    }
    free_graph(dev);
    dev->dirty = false;
    return DPV_OK;
}

// Issue one frame's launches on stream `st`: ray setup and culling, the
// brick ray-march, the sort-last composite.  Stage timers are recorded only
// when `timed` (not while capturing a graph).
dpv_status enqueue_render(dpv_device dev, cudaStream_t st, bool timed) {
    const FrameParams& P = dev->P;
    float3 og = make_float3(dev->origin[0], dev->origin[1], dev->origin[2]);
    const bool iso = P.iso_on != 0;
    const bool ordered = P.ordered_on != 0;
    const bool persistent = (dev->frame.flags & DPV_FRAME_PERSISTENT) && !(dev->frame.flags & DPV_FRAME_STAGED) &&
                            !iso && !ordered;
    CK(cudaMemsetAsync(dev->d_counters, 0, sizeof(Counters), st), "reset counters");
    cudaEvent_t t0 = timed ? stage_start(dev) : nullptr;
    CK(launch_cull(P, dev->d_cam_in, og, dev->spacing, dev->d_cams, dev->d_camd, dev->d_rays, dev->d_bricks,
                   dev->d_rects, dev->d_tile_count, dev->d_tile_first, dev->d_items, dev->items_cap, dev->d_counters,
                   true, st),
       "cull");
    Schedule sch{dev->d_sched, dev->d_work, 0};
    if (persistent || P.shadow_on)
        CK(launch_schedule(P, dev->d_items, dev->n_items, 1, dev->d_hist, dev->d_offsets, dev->d_cursor,
                           dev->d_tmp64, dev->d_sched, st),
           "schedule");
    if (P.skip_on)
        CK(launch_classify_empty(dev->bricks[0].dtype, P, dev->d_bricks, dev->nranks, dev->d_scales, dev->max_macro,
                                 dev->d_tf, dev->d_tfz, st),
           "macro-cell transparency");
    if (timed) stage_stop(dev, DPV_STAGE_CULL, t0);
    t0 = timed ? stage_start(dev) : nullptr;
    if (ordered) {
        // march and composite in one launch: the frame is written directly
        // (the persistent form when DPV_FRAME_PERSISTENT is set)
        const bool pers_ord = (dev->frame.flags & DPV_FRAME_PERSISTENT) != 0;
        CK(launch_march_ordered(dev->bricks[0].dtype, dev->gather, P, dev->d_cams, dev->d_bricks, dev->d_scales,
                                dev->d_tile_first, dev->d_tile_count, dev->d_items, dev->d_tf, dev->d_out_rgba,
                                dev->d_out_depth, P.order_stride ? dev->d_order : nullptr, dev->d_counters,
                                pers_ord ? dev->d_work : nullptr, st),
           "ordered march");
        if (timed) stage_stop(dev, DPV_STAGE_MARCH, t0);
        dev->launches += 6 + 1;
        return DPV_OK;
    }
    if (P.shadow_on) {
        // shadow rays: records per slot, spawn, the forwarding rounds, the
        // shading march (fragments as the sort-last march writes them)
        CK(launch_shadow_offsets(P, dev->d_cams, dev->d_bricks, dev->d_items, dev->n_items, dev->d_sched,
                                 dev->d_sh_counts, dev->d_sh_offsets, dev->d_sh_chunks, dev->d_sh_total, st),
           "shadow offsets");
        CK(launch_shadow_render(dev->bricks[0].dtype, dev->gather, P, dev->d_cams, dev->d_bricks, dev->d_scales,
                                dev->d_items, dev->n_items, dev->d_sched, dev->d_offsets, dev->d_sh_offsets,
                                dev->d_sh_total, dev->d_rec_first, dev->n_recs, dev->d_recs, dev->d_tf,
                                dev->d_frag_rgba, dev->d_frag_key, dev->d_counters, st),
           "shadow march");
        dev->launches += 4 + 2 + P.nbricks + 1;
    } else if (iso)
        CK(launch_iso_fwd(dev->bricks[0].dtype, dev->gather, P, dev->d_cams, dev->d_bricks, dev->d_scales,
                          dev->d_items, dev->n_items, dev->d_tf, dev->d_frag_rgba, dev->d_frag_key, dev->d_counters,
                          st),
           "iso march");
    else if (!(dev->frame.flags & DPV_FRAME_STAGED))
        CK(launch_march_fwd(dev->bricks[0].dtype, dev->gather, P, dev->d_cams, dev->d_bricks, dev->d_scales,
                            dev->d_items, dev->n_items, dev->d_tf, dev->d_frag_rgba, dev->d_frag_key, dev->d_counters,
                            st, persistent ? &sch : nullptr),
           "march");
    else
        CK(launch_march_fwd_staged(dev->bricks[0].dtype, P, dev->d_cams, dev->d_bricks, dev->d_scales, dev->d_items,
                                   dev->n_items, dev->d_tf, dev->d_frag_rgba, dev->d_frag_key, dev->d_counters, st),
           "march");
    if (timed) stage_stop(dev, DPV_STAGE_MARCH, t0);
    t0 = timed ? stage_start(dev) : nullptr;
    if (iso)
        CK(launch_composite_iso(P, dev->d_cams, dev->d_tile_first, dev->d_tile_count, dev->d_items, dev->d_frag_rgba,
                                dev->d_frag_key, dev->d_out_rgba, dev->d_out_depth,
                                P.order_stride ? dev->d_order : nullptr, st),
           "composite");
    else
        CK(launch_composite_fwd(P, 1.0f / dev->spacing, dev->d_cams, dev->d_tile_first, dev->d_tile_count,
                                dev->d_items, dev->d_frag_rgba, dev->d_frag_key, dev->d_out_rgba, dev->d_out_depth,
                                P.order_stride ? dev->d_order : nullptr, st),
           "composite");
    if (timed) stage_stop(dev, DPV_STAGE_COMPOSITE, t0);
    dev->launches += 6 + (persistent || P.shadow_on ? 3 : 0) + (dev->n_items > 0 && !P.shadow_on ? 1 : 0) + 1;
    return DPV_OK;
}

// Capture the per-frame launches into a graph (once per prepared frame).
// On a capture failure the device falls back to direct launches.
void ensure_graph(dpv_device dev) {
    if (dev->graph || dev->graph_failed) return;
    if (!dev->cap_stream && cudaStreamCreateWithFlags(&dev->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        dev->graph_failed = true;
        return;
    }
    cudaGraph_t g = nullptr;
    uint64_t launches = dev->launches;
    if (cudaStreamBeginCapture(dev->cap_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        cudaGetLastError();
        dev->graph_failed = true;
        return;
    }
    dpv_status s = enqueue_render(dev, dev->cap_stream, false);
    cudaError_t e = cudaStreamEndCapture(dev->cap_stream, &g);
    dev->launches = launches;
    if (s != DPV_OK || e != cudaSuccess || !g) {
        cudaGetLastError();
        dev->poisoned = false;                // a failed capture issued no work
        if (g) cudaGraphDestroy(g);
        dev->graph_failed = true;
        return;
    }
    e = cudaGraphInstantiate(&dev->graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        cudaGetLastError();
        dev->graph = nullptr;
        dev->graph_failed = true;
    }
}

}  // namespace

extern "C" {

const char* dpvGetLastError(void) { return g_last_error.c_str(); }

dpv_status dpvCreateDevice(int num_ranks, int cuda_device, void* cuda_stream, dpv_device* out) {
    g_last_error.clear();
    if (!out) return fail(DPV_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (num_ranks < 1 || num_ranks > MAX_RANKS) return fail(DPV_ERR_INVALID_ARG, "num_ranks must be 1..%d", MAX_RANKS);
    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess) return fail(DPV_ERR_CUDA, "no CUDA device: %s", cudaGetErrorString(e));
    if (cuda_device < 0 || cuda_device >= ndev) return fail(DPV_ERR_INVALID_ARG, "cuda_device %d out of range", cuda_device);
    dpv_device dev = new (std::nothrow) dpv_device_t();
    if (!dev) return fail(DPV_ERR_OUT_OF_MEMORY, "host allocation failed");
    dev->nranks = num_ranks;
    dev->cuda_device = cuda_device;
    dev->stream = (cudaStream_t)cuda_stream;
    dev->bricks.resize(num_ranks);
    DeviceGuard g(cuda_device);
    dpv_status s;
    if ((s = dev_alloc(dev, (void**)&dev->d_scales, sizeof(float) * MAX_RANKS, "scales")) ||
        (s = dev_alloc(dev, (void**)&dev->d_tmp, sizeof(unsigned int) * 4, "scratch"))) {
        dpvRelease(dev);
        return s;
    }
    e = cudaEventCreateWithFlags(&dev->ev_done, cudaEventDisableTiming);
    if (e != cudaSuccess) {
        dpvRelease(dev);
        return fail(DPV_ERR_CUDA, "event: %s", cudaGetErrorString(e));
    }
    *out = dev;
    return DPV_OK;
}

dpv_status dpvSetVolumeGeometry(dpv_device dev, const int dims[3], const float origin[3], float spacing) {
    dpv_status s = check_dev(dev);
    if (s) return s;
    if (!dims || !origin) return fail(DPV_ERR_INVALID_ARG, "dims/origin NULL");
    for (int a = 0; a < 3; ++a)
        if (dims[a] < 2) return fail(DPV_ERR_INVALID_ARG, "dims[%d] = %d < 2", a, dims[a]);
    if (!(spacing > 0.0f) || !isfinite(spacing)) return fail(DPV_ERR_INVALID_ARG, "spacing must be > 0");
    DeviceGuard g(dev->cuda_device);
    for (auto& b : dev->bricks) {
        dev_free(b.data);
        dev_free(b.gather);
        dev_free(b.mm);
        b = HostBrick();
    }
    for (int a = 0; a < 3; ++a) {
        dev->dims[a] = dims[a];
        dev->origin[a] = origin[a];
    }
    dev->spacing = spacing;
    dev->has_geom = true;
    dev->dirty = true;
    return DPV_OK;
}

dpv_status dpvCommitBrick(dpv_device dev, int rank, const dpv_brick_desc* d) {
    dpv_status s = check_dev(dev);
    if (s) return s;
    if (!dev->has_geom) return fail(DPV_ERR_STATE, "set the volume geometry before committing bricks");
    if (rank < 0 || rank >= dev->nranks) return fail(DPV_ERR_INVALID_ARG, "rank %d out of range", rank);
    if (!d || !d->data) return fail(DPV_ERR_INVALID_ARG, "brick descriptor or data is NULL");
    if ((int)d->storage < 0 || (int)d->storage > 3 || (int)d->src_dtype < 0 || (int)d->src_dtype > 3)
        return fail(DPV_ERR_INVALID_ARG, "bad dtype");
    if (d->src_dtype != DPV_F32 && d->src_dtype != d->storage)
        return fail(DPV_ERR_UNSUPPORTED, "source data must be float32 or already in the storage format");
    HostBrick nb;
    long long nodes = 1;
    for (int a = 0; a < 3; ++a) {
        if (d->owned_lo[a] < 0 || d->owned_hi[a] > dev->dims[a] || d->owned_lo[a] >= d->owned_hi[a])
            return fail(DPV_ERR_INVALID_ARG, "owned range on axis %d is [%d, %d) in a volume of %d nodes", a,
                        d->owned_lo[a], d->owned_hi[a], dev->dims[a]);
        nb.lo[a] = d->owned_lo[a];
        nb.hi[a] = d->owned_hi[a];
        nb.s_lo[a] = std::max(d->owned_lo[a] - 1, 0);
        int s_hi = std::min(d->owned_hi[a], dev->dims[a] - 1);
        nb.s_n[a] = s_hi - nb.s_lo[a] + 1;
        nodes *= nb.s_n[a];
        if (d->data_dims[a] < 1 || d->data_lo[a] > nb.s_lo[a] || d->data_lo[a] + d->data_dims[a] < nb.s_lo[a] + nb.s_n[a])
            return fail(DPV_ERR_INVALID_ARG, "data box on axis %d does not contain the stored nodes [%d, %d)", a,
                        nb.s_lo[a], nb.s_lo[a] + nb.s_n[a]);
    }
    if (nodes > 0x7fffffffLL) return fail(DPV_ERR_UNSUPPORTED, "brick stores %lld nodes (max 2^31 - 1)", nodes);
    nb.dtype = (int)d->storage;
    nb.bytes = (size_t)nodes * kElemSize[nb.dtype];
    DeviceGuard g(dev->cuda_device);
    HostBrick& hb = dev->bricks[rank];
    if (hb.data && hb.bytes == nb.bytes) {
        nb.data = hb.data;
        hb.data = nullptr;
    } else {
        dev_free(hb.data);
        hb.data = nullptr;
        if ((s = dev_alloc(dev, &nb.data, nb.bytes, "brick storage"))) return s;
    }
    CommitArgs a;
    void* staging = nullptr;
    if (d->data_on_device) {
        a.src = d->data;
        for (int k = 0; k < 3; ++k) {
            a.d_lo[k] = d->data_lo[k];
            a.d_n[k] = d->data_dims[k];
        }
    } else {
        // copy just the stored box from the host into a staging buffer
        size_t es = kElemSize[d->src_dtype];
        if ((s = dev_alloc(dev, &staging, (size_t)nodes * es, "staging"))) {
            dev_free(nb.data);
            return s;
        }
        cudaMemcpy3DParms p;
        memset(&p, 0, sizeof p);
        p.srcPtr = make_cudaPitchedPtr((void*)d->data, (size_t)d->data_dims[0] * es, (size_t)d->data_dims[0],
                                       (size_t)d->data_dims[1]);
        p.srcPos = make_cudaPos((size_t)(nb.s_lo[0] - d->data_lo[0]) * es, (size_t)(nb.s_lo[1] - d->data_lo[1]),
                                (size_t)(nb.s_lo[2] - d->data_lo[2]));
        p.dstPtr = make_cudaPitchedPtr(staging, (size_t)nb.s_n[0] * es, (size_t)nb.s_n[0], (size_t)nb.s_n[1]);
        p.extent = make_cudaExtent((size_t)nb.s_n[0] * es, (size_t)nb.s_n[1], (size_t)nb.s_n[2]);
        p.kind = cudaMemcpyHostToDevice;
        CK(cudaMemcpy3DAsync(&p, dev->stream), "copy brick from host");
        a.src = staging;
        for (int k = 0; k < 3; ++k) {
            a.d_lo[k] = nb.s_lo[k];
            a.d_n[k] = nb.s_n[k];
        }
    }
    for (int k = 0; k < 3; ++k) {
        a.s_lo[k] = nb.s_lo[k];
        a.s_n[k] = nb.s_n[k];
    }
    cudaError_t e = launch_commit(a, nb.dtype, d->src_dtype == DPV_F32, d->scale, dev->d_tmp, dev->d_scales + rank,
                                  nb.data, dev->stream);
    if (staging) {
        cudaError_t e2 = cudaStreamSynchronize(dev->stream);
        dev_free(staging);
        if (e == cudaSuccess) e = e2;
    }
    if (e != cudaSuccess) return cuda_fail(dev, e, "brick commit");
    nb.committed = true;
    nb.gather = hb.gather;              // the gather layout is rebuilt at the next render
    nb.gather_bytes = hb.gather_bytes;
    nb.gather_kind = hb.gather_kind;
    nb.gather_valid = false;
    nb.mm = hb.mm;                      // value ranges too
    nb.mm_cells = hb.mm_cells;
    nb.mm_valid = false;
    hb = nb;
    dev->dirty = true;
    return DPV_OK;
}

dpv_status dpvSetTransferFunction(dpv_device dev, const float* rgba, int n, float vmin, float vmax, int on_device) {
    dpv_status s = check_dev(dev);
    if (s) return s;
    if (!rgba) return fail(DPV_ERR_INVALID_ARG, "rgba is NULL");
    if (n < 2 || n > MAX_TF) return fail(DPV_ERR_INVALID_ARG, "TF size %d not in 2..%d", n, MAX_TF);
    if (!(vmax > vmin)) return fail(DPV_ERR_INVALID_ARG, "need vmax > vmin");
    DeviceGuard g(dev->cuda_device);
    if (n > dev->ntf || !dev->d_tf) {
        dev_free(dev->d_tf);
        dev->d_tf = nullptr;
        if ((s = dev_alloc(dev, (void**)&dev->d_tf, sizeof(float4) * n, "TF"))) return s;
    }
    if (on_device) {
        CK(cudaMemcpyAsync(dev->d_tf, rgba, sizeof(float4) * n, cudaMemcpyDeviceToDevice, dev->stream), "upload TF");
    } else {
        const int k = dev->tf_stage_next;
        dev->tf_stage_next ^= 1;
        if (!dev->h_tf_stage[k]) {
            CK(cudaHostAlloc((void**)&dev->h_tf_stage[k], sizeof(float4) * MAX_TF, cudaHostAllocDefault),
               "TF staging");
            CK(cudaEventCreateWithFlags(&dev->ev_tf_stage[k], cudaEventDisableTiming), "TF staging");
        } else {
            CK(cudaEventSynchronize(dev->ev_tf_stage[k]), "TF staging");   // its last upload has run
        }
        memcpy(dev->h_tf_stage[k], rgba, sizeof(float4) * n);
        CK(cudaMemcpyAsync(dev->d_tf, dev->h_tf_stage[k], sizeof(float4) * n, cudaMemcpyHostToDevice, dev->stream),
           "upload TF");
        CK(cudaEventRecord(dev->ev_tf_stage[k], dev->stream), "upload TF");
    }
    if (n != dev->ntf || vmin != dev->vmin || vmax != dev->vmax) dev->dirty = true;
    dev->ntf = n;
    dev->vmin = vmin;
    dev->vmax = vmax;
    return DPV_OK;
}

dpv_status dpvSetLight(dpv_device dev, const float direction[3], float step_voxels, float ambient) {
    dpv_status s = check_dev(dev);
    if (s) return s;
    if (!direction) return fail(DPV_ERR_INVALID_ARG, "direction is NULL");
    const double x = direction[0], y = direction[1], z = direction[2];
    const double n = std::sqrt(x * x + y * y + z * z);
    if (!(n > 0.0) || !std::isfinite(n)) return fail(DPV_ERR_INVALID_ARG, "light direction must be finite, non-zero");
    if (!(step_voxels >= 1.0f / 64.0f && step_voxels <= 64.0f))
        return fail(DPV_ERR_INVALID_ARG, "shadow step %g not in [1/64, 64] voxels", (double)step_voxels);
    if (!(ambient >= 0.0f && ambient <= 1.0f)) return fail(DPV_ERR_INVALID_ARG, "ambient not in [0, 1]");
    dev->light_dir[0] = (float)(x / n);
    dev->light_dir[1] = (float)(y / n);
    dev->light_dir[2] = (float)(z / n);
    dev->light_step = step_voxels;
    dev->light_ambient = ambient;
    dev->has_light = true;
    dev->dirty = true;
    return DPV_OK;
}

dpv_status dpvSetCameras(dpv_device dev, const dpv_camera* cams, int n) {
    dpv_status s = check_dev(dev);
    if (s) return s;
    if (!cams || n < 1) return fail(DPV_ERR_INVALID_ARG, "need at least one camera");
    std::vector<CamIn> v(n);
    for (int i = 0; i < n; ++i) {
        const dpv_camera& c = cams[i];
        if (const char* why = camera_problem(c)) return fail(DPV_ERR_INVALID_ARG, "camera %d: %s", i, why);
        memcpy(&v[i], &c, sizeof(CamIn));
    }
    dev->cams.swap(v);
    dev->dirty = true;
    return DPV_OK;
}

dpv_status dpvSetFrame(dpv_device dev, const dpv_frame_desc* f) {
    dpv_status s = check_dev(dev);
    if (s) return s;
    if (!f) return fail(DPV_ERR_INVALID_ARG, "frame descriptor is NULL");
    if (f->width < 1 || f->height < 1) return fail(DPV_ERR_INVALID_ARG, "frame size %dx%d", f->width, f->height);
    if (!(f->step_voxels > 0.0f)) return fail(DPV_ERR_INVALID_ARG, "step_voxels must be > 0");
    if (!(f->sigma_max >= 0.0f)) return fail(DPV_ERR_INVALID_ARG, "sigma_max must be >= 0");
    int tw = f->tile_w > 0 ? f->tile_w : 16, th = f->tile_h > 0 ? f->tile_h : 16;
    if (tw % 8 || th % 4 || tw * th > 256)
        return fail(DPV_ERR_INVALID_ARG, "tile %dx%d: width a multiple of 8, height of 4, at most 256 pixels", tw, th);
    if ((f->flags & DPV_FRAME_ISO) && (f->flags & DPV_FRAME_STAGED))
        return fail(DPV_ERR_UNSUPPORTED, "iso-surface frames have no staged form");
    if ((f->flags & DPV_FRAME_ORDERED) && (f->flags & (DPV_FRAME_STAGED | DPV_FRAME_ISO)))
        return fail(DPV_ERR_UNSUPPORTED, "the ordered march has no staged or iso-surface form");
    if ((f->flags & DPV_FRAME_SKIP) && (f->flags & (DPV_FRAME_STAGED | DPV_FRAME_ISO)))
        return fail(DPV_ERR_UNSUPPORTED, "empty-space skipping has no staged or iso-surface form");
    if ((f->flags & DPV_FRAME_DEEP) && (f->flags & (DPV_FRAME_STAGED | DPV_FRAME_ISO | DPV_FRAME_ORDERED)))
        return fail(DPV_ERR_UNSUPPORTED, "deep fragments have no staged, iso-surface or ordered form");
    if ((f->flags & DPV_FRAME_SHADOW) &&
        (f->flags & (DPV_FRAME_STAGED | DPV_FRAME_ISO | DPV_FRAME_ORDERED | DPV_FRAME_SKIP | DPV_FRAME_DEEP)))
        return fail(DPV_ERR_UNSUPPORTED, "shadows have no staged, iso-surface, ordered, skipping or deep form");
    if ((f->flags & DPV_FRAME_ISO) && !isfinite(f->iso_value))
        return fail(DPV_ERR_INVALID_ARG, "iso_value must be finite");
    dev->frame = *f;
    dev->has_frame = true;
    dev->dirty = true;
    return DPV_OK;
}

dpv_status dpvRenderFrame(dpv_device dev) {
    dpv_status s = check_dev(dev);
    if (s) return s;
    if (!dev->has_geom) return fail(DPV_ERR_STATE, "no volume geometry");
    for (int k = 0; k < dev->nranks; ++k)
        if (!dev->bricks[k].committed) return fail(DPV_ERR_STATE, "rank %d has not committed its brick", k);
    if (!dev->d_tf) return fail(DPV_ERR_STATE, "no transfer function");
    if (dev->cams.empty()) return fail(DPV_ERR_STATE, "no cameras");
    if (!dev->has_frame) return fail(DPV_ERR_STATE, "no frame parameters");
    DeviceGuard g(dev->cuda_device);
    if (dev->dirty) {
        if ((s = check_partition(dev))) return s;
        if ((s = prepare(dev))) return s;
    }
    if ((dev->frame.flags & DPV_FRAME_GRAPH) && !dev->profiling) {
        ensure_graph(dev);
        if (dev->graph) {
            CK(cudaGraphLaunch(dev->graph, dev->stream), "graph launch");
            ++dev->graph_launches;
            dev->launches += 6 + ((dev->frame.flags & DPV_FRAME_PERSISTENT) ? 3 : 0) + (dev->n_items > 0 ? 1 : 0) + 1;
        } else if ((s = enqueue_render(dev, dev->stream, true))) {
            return s;
        }
    } else if ((s = enqueue_render(dev, dev->stream, true))) {
        return s;
    }
    CK(cudaEventRecord(dev->ev_done, dev->stream), "record");
    dev->rendered = true;
    return DPV_OK;
}

dpv_status dpvFrameReady(dpv_device dev, int wait, int* ready) {
    dpv_status s = check_dev(dev);
    if (s) return s;
    if (!ready) return fail(DPV_ERR_INVALID_ARG, "ready is NULL");
    if (!dev->rendered) {
        *ready = 1;
        return DPV_OK;
    }
    DeviceGuard g(dev->cuda_device);
    cudaError_t e = wait ? cudaEventSynchronize(dev->ev_done) : cudaEventQuery(dev->ev_done);
    if (e == cudaErrorNotReady) {
        *ready = 0;
        return DPV_OK;
    }
    if (e != cudaSuccess) return cuda_fail(dev, e, "frame completion");
    *ready = 1;
    return DPV_OK;
}

dpv_status dpvMapFrame(dpv_device dev, int camera, const float** rgba, const float** depth) {
    dpv_status s = check_dev(dev);
    if (s) return s;
    if (!dev->rendered) return fail(DPV_ERR_STATE, "no frame rendered yet");
    if (camera < 0 || camera >= dev->P.ncam) return fail(DPV_ERR_INVALID_ARG, "camera %d out of range", camera);
    size_t off = (size_t)camera * dev->P.W * dev->P.H;
    if (rgba) *rgba = (const float*)(dev->d_out_rgba + off);
    if (depth) *depth = dev->d_out_depth + off;
    return DPV_OK;
}

dpv_status dpvUnmapFrame(dpv_device dev, int camera) {
    dpv_status s = check_dev(dev);
    if (s) return s;
    if (camera < 0 || camera >= dev->P.ncam) return fail(DPV_ERR_INVALID_ARG, "camera %d out of range", camera);
    return DPV_OK;
}

dpv_status dpvCopyFrame(dpv_device dev, int camera, float* rgba, float* depth) {
    const float *r = nullptr, *d = nullptr;
    dpv_status s = dpvMapFrame(dev, camera, &r, &d);
    if (s) return s;
    DeviceGuard g(dev->cuda_device);
    size_t n = (size_t)dev->P.W * dev->P.H;
    if (rgba) CK(cudaMemcpyAsync(rgba, r, n * sizeof(float4), cudaMemcpyDefault, dev->stream), "copy frame");
    if (depth) CK(cudaMemcpyAsync(depth, d, n * sizeof(float), cudaMemcpyDefault, dev->stream), "copy frame");
    cudaPointerAttributes at;
    bool host = false;
    if (rgba && cudaPointerGetAttributes(&at, rgba) == cudaSuccess && at.type != cudaMemoryTypeDevice &&
        at.type != cudaMemoryTypeManaged)
        host = true;
    if (depth && cudaPointerGetAttributes(&at, depth) == cudaSuccess && at.type != cudaMemoryTypeDevice &&
        at.type != cudaMemoryTypeManaged)
        host = true;
    cudaGetLastError();
    if (host) CK(cudaStreamSynchronize(dev->stream), "copy frame");
    return DPV_OK;
}

dpv_status dpvCopyFrameAsync(dpv_device dev, int camera, float* rgba, float* depth) {
    dpv_status s = check_dev(dev);
    if (s) return s;
    if (!dev->rendered) return fail(DPV_ERR_STATE, "no frame rendered yet");
    if (camera < -1 || camera >= dev->P.ncam) return fail(DPV_ERR_INVALID_ARG, "camera %d out of range", camera);
    DeviceGuard g(dev->cuda_device);
    const size_t per = (size_t)dev->P.W * dev->P.H;
    const size_t n = camera < 0 ? per * dev->P.ncam : per;
    const size_t off = camera < 0 ? 0 : per * camera;
    if (!dev->copy_stream) {
        CK(cudaStreamCreateWithFlags(&dev->copy_stream, cudaStreamNonBlocking), "copy stream");
        for (int k = 0; k < 2; ++k) {
            CK(cudaEventCreateWithFlags(&dev->ev_staged[k], cudaEventDisableTiming), "copy events");
            CK(cudaEventCreateWithFlags(&dev->ev_drained[k], cudaEventDisableTiming), "copy events");
        }
    }
    if (n > dev->stage_cap) {
        CK(cudaStreamSynchronize(dev->copy_stream), "copy stream");
        for (int k = 0; k < 2; ++k) {
            dev_free(dev->d_stage_rgba[k]);
            dev_free(dev->d_stage_depth[k]);
            dev->d_stage_rgba[k] = nullptr;
            dev->d_stage_depth[k] = nullptr;
        }
        dev->stage_cap = 0;
        for (int k = 0; k < 2; ++k) {
            if ((s = dev_alloc(dev, (void**)&dev->d_stage_rgba[k], sizeof(float4) * n, "copy staging"))) return s;
            if ((s = dev_alloc(dev, (void**)&dev->d_stage_depth[k], sizeof(float) * n, "copy staging"))) return s;
        }
        dev->stage_cap = n;
    }
    const int k = dev->stage_next;
    dev->stage_next ^= 1;
    // the slot's previous drain must be done before the device stream
    // overwrites it; the drain then runs beside the next render
    CK(cudaStreamWaitEvent(dev->stream, dev->ev_drained[k], 0), "copy order");
    if (rgba)
        CK(cudaMemcpyAsync(dev->d_stage_rgba[k], dev->d_out_rgba + off, sizeof(float4) * n, cudaMemcpyDeviceToDevice,
                           dev->stream),
           "stage frame");
    if (depth)
        CK(cudaMemcpyAsync(dev->d_stage_depth[k], dev->d_out_depth + off, sizeof(float) * n,
                           cudaMemcpyDeviceToDevice, dev->stream),
           "stage frame");
    CK(cudaEventRecord(dev->ev_staged[k], dev->stream), "copy order");
    CK(cudaStreamWaitEvent(dev->copy_stream, dev->ev_staged[k], 0), "copy order");
    if (rgba)
        CK(cudaMemcpyAsync(rgba, dev->d_stage_rgba[k], sizeof(float4) * n, cudaMemcpyDefault, dev->copy_stream),
           "copy frame");
    if (depth)
        CK(cudaMemcpyAsync(depth, dev->d_stage_depth[k], sizeof(float) * n, cudaMemcpyDefault, dev->copy_stream),
           "copy frame");
    CK(cudaEventRecord(dev->ev_drained[k], dev->copy_stream), "copy order");
    return DPV_OK;
}

dpv_status dpvCopyWait(dpv_device dev) {
    dpv_status s = check_dev(dev);
    if (s) return s;
    if (!dev->copy_stream) return DPV_OK;
    DeviceGuard g(dev->cuda_device);
    CK(cudaStreamSynchronize(dev->copy_stream), "copy wait");
    return DPV_OK;
}

dpv_status dpvReadDeepFragments(dpv_device dev, int camera, int rank, int layer, float* rgba, int32_t* key) {
    dpv_status s = check_dev(dev);
    if (s) return s;
    if (!dev->rendered) return fail(DPV_ERR_STATE, "no frame rendered yet");
    if (camera < 0 || camera >= dev->P.ncam) return fail(DPV_ERR_INVALID_ARG, "camera %d out of range", camera);
    if (rank < 0 || rank >= dev->nranks) return fail(DPV_ERR_INVALID_ARG, "rank %d out of range", rank);
    if (layer < 0 || layer >= dev->P.deep)
        return fail(DPV_ERR_INVALID_ARG, "layer %d out of range (the frame has %d)", layer, dev->P.deep);
    if (!rgba || !key) return fail(DPV_ERR_INVALID_ARG, "output NULL");
    DeviceGuard g(dev->cuda_device);
    CK(launch_read_frags(dev->P, dev->d_items, dev->n_items, camera, rank, layer, dev->d_frag_rgba, dev->d_frag_key,
                         (float4*)rgba, key, dev->stream),
       "read fragments");
    return DPV_OK;
}

dpv_status dpvReadFragments(dpv_device dev, int camera, int rank, float* rgba, int32_t* key) {
    return dpvReadDeepFragments(dev, camera, rank, 0, rgba, key);
}

dpv_status dpvMapFragments(dpv_device dev, int camera, int rank, const void** frag) {
    dpv_status s = check_dev(dev);
    if (s) return s;
    if (!dev->rendered) return fail(DPV_ERR_STATE, "no frame rendered yet");
    if (camera < 0 || camera >= dev->P.ncam) return fail(DPV_ERR_INVALID_ARG, "camera %d out of range", camera);
    if (rank < 0 || rank >= dev->nranks) return fail(DPV_ERR_INVALID_ARG, "rank %d out of range", rank);
    if (!frag) return fail(DPV_ERR_INVALID_ARG, "frag is NULL");
    DeviceGuard g(dev->cuda_device);
    const size_t npix = (size_t)dev->P.W * dev->P.H;
    const size_t bytes = npix * (sizeof(float4) + sizeof(int32_t));
    const long long key = (long long)camera * (MAX_RANKS + 1) + rank;
    auto it = dev->frag_maps.find(key);
    if (it != dev->frag_maps.end() && it->second.bytes != bytes) {
        CK(cudaStreamSynchronize(dev->stream), "remap fragments");
        dev_free(it->second.ptr);
        dev->frag_maps.erase(it);
        it = dev->frag_maps.end();
    }
    if (it == dev->frag_maps.end()) {
        void* p = nullptr;
        if ((s = dev_alloc(dev, &p, bytes, "mapped fragments"))) return s;
        it = dev->frag_maps.emplace(key, dpv_device_t::FragMap{p, bytes}).first;
    }
    float4* rgba = (float4*)it->second.ptr;
    int* keys = (int*)(rgba + npix);
    CK(launch_read_frags(dev->P, dev->d_items, dev->n_items, camera, rank, 0, dev->d_frag_rgba, dev->d_frag_key,
                         rgba, keys, dev->stream),
       "map fragments");
    *frag = it->second.ptr;
    return DPV_OK;
}

dpv_status dpvUnmapFragments(dpv_device dev, int camera, int rank) {
    dpv_status s = check_dev(dev);
    if (s) return s;
    const long long key = (long long)camera * (MAX_RANKS + 1) + rank;
    auto it = dev->frag_maps.find(key);
    if (it == dev->frag_maps.end())
        return fail(DPV_ERR_STATE, "fragments of camera %d, rank %d are not mapped", camera, rank);
    DeviceGuard g(dev->cuda_device);
    CK(cudaStreamSynchronize(dev->stream), "unmap fragments");
    dev_free(it->second.ptr);
    dev->frag_maps.erase(it);
    return DPV_OK;
}

dpv_status dpvReadBrick(dpv_device dev, int rank, void* dst, int stored_lo[3], int stored_dims[3], float* scale) {
    dpv_status s = check_dev(dev);
    if (s) return s;
    if (rank < 0 || rank >= dev->nranks) return fail(DPV_ERR_INVALID_ARG, "rank %d out of range", rank);
    const HostBrick& b = dev->bricks[rank];
    if (!b.committed) return fail(DPV_ERR_STATE, "rank %d has not committed its brick", rank);
    DeviceGuard g(dev->cuda_device);
    if (dst) CK(cudaMemcpyAsync(dst, b.data, b.bytes, cudaMemcpyDeviceToDevice, dev->stream), "read brick");
    float sc = 1.0f;
    CK(cudaMemcpyAsync(&sc, dev->d_scales + rank, sizeof(float), cudaMemcpyDeviceToHost, dev->stream), "read scale");
    CK(cudaStreamSynchronize(dev->stream), "read brick");
    for (int a = 0; a < 3; ++a) {
        if (stored_lo) stored_lo[a] = b.s_lo[a];
        if (stored_dims) stored_dims[a] = b.s_n[a];
    }
    if (scale) *scale = sc;
    return DPV_OK;
}

dpv_status dpvMapOrder(dpv_device dev, int camera, const uint8_t** order, int* stride) {
    dpv_status s = check_dev(dev);
    if (s) return s;
    if (!dev->rendered) return fail(DPV_ERR_STATE, "no frame rendered yet");
    if (!dev->P.order_stride) return fail(DPV_ERR_STATE, "frame was rendered without DPV_FRAME_ORDER");
    if (camera < 0 || camera >= dev->P.ncam) return fail(DPV_ERR_INVALID_ARG, "camera %d out of range", camera);
    if (!order || !stride) return fail(DPV_ERR_INVALID_ARG, "output NULL");
    *order = dev->d_order + (size_t)camera * dev->P.W * dev->P.H * dev->P.order_stride;
    *stride = dev->P.order_stride;
    return DPV_OK;
}

namespace {
dpv_status finish_backward(dpv_device dev) {
    dev->launches += 1;   // the compositor's adjoint
    return DPV_OK;
}
}  // namespace

dpv_status dpvBackward(dpv_device dev, const float* dL_drgba, double* dL_dtf, float* dL_dvol) {
    dpv_status s = check_dev(dev);
    if (s) return s;
    if (!dev->rendered || dev->dirty) return fail(DPV_ERR_STATE, "backward needs the fragments of a render");
    if (dev->P.iso_on) return fail(DPV_ERR_UNSUPPORTED, "the adjoint is of the volume-rendering mode");
    if (dev->P.ordered_on) return fail(DPV_ERR_UNSUPPORTED, "the adjoint is of the sort-last march");
    if (dev->P.deep > 1) return fail(DPV_ERR_UNSUPPORTED, "the adjoint is of one fragment per brick");
    if (dev->P.shadow_on) return fail(DPV_ERR_UNSUPPORTED, "the adjoint is of the unshadowed march");
    if (!dL_drgba || !dL_dtf) return fail(DPV_ERR_INVALID_ARG, "gradient pointers NULL");
    DeviceGuard g(dev->cuda_device);
    const FrameParams& P = dev->P;
    if (!dev->d_frag_grad) {
        if ((s = dev_alloc(dev, (void**)&dev->d_frag_grad, sizeof(float4) * dev->frag_cap * P.tp, "fragment grads")))
            return s;
    }
    CK(cudaMemsetAsync(dL_dtf, 0, sizeof(double) * 4 * dev->ntf, dev->stream), "zero dtf");
    // field gradient: through the face adjoint buffer (two vector reductions
    // per sample, then a gather that writes every node) where the slots of
    // the largest brick fit in half of the free device memory.  Where the
    // whole buffer does not fit, the bricks are taken in groups of
    // consecutive ranks whose slots fit: each group's items are replayed,
    // then its slots are gathered and added into the field.
    // DPV_FACE_GRAD=0 selects the scalar atomics into the field instead;
    // DPV_FACE_GROUP=n takes at most n bricks per group.
    const bool staged = (dev->frame.flags & DPV_FRAME_STAGED) != 0;
    bool faces = dL_dvol && !staged && dev->gface_slots > 0;
    if (faces) {
        if (const char* env = getenv("DPV_FACE_GRAD")) faces = atoi(env) != 0;
    }
    const size_t want = dev->gface_slots;
    int group_max = dev->nranks;
    if (const char* env = getenv("DPV_FACE_GROUP")) {
        int v = atoi(env);
        if (v > 0 && v < group_max) group_max = v;
    }
    size_t max_brick = 0;
    for (int k = 0; k < dev->nranks; ++k)
        max_brick = std::max(max_brick, dev->gface_off_h[k + 1] - dev->gface_off_h[k]);
    if (faces && dev->gface_cap < want && dev->gface_tried != want) {
        dev_free(dev->d_gface);
        dev->d_gface = nullptr;
        dev->gface_cap = 0;
        dev->gface_tried = want;
        size_t free_b = 0, total_b = 0;
        cudaMemGetInfo(&free_b, &total_b);
        size_t n = std::min(want, free_b / 2 / sizeof(float4));
        if (n >= max_brick && cudaMalloc((void**)&dev->d_gface, n * sizeof(float4)) == cudaSuccess)
            dev->gface_cap = n;
        else
            cudaGetLastError();
    }
    faces = faces && dev->d_gface && dev->gface_cap >= max_brick;
    // groups [grp[i], grp[i + 1]) of consecutive ranks
    std::vector<int> grp{0};
    if (faces) {
        for (int k = 0; k < dev->nranks; ++k) {
            const bool full = dev->gface_off_h[k + 1] - dev->gface_off_h[grp.back()] > dev->gface_cap;
            if (full || k - grp.back() >= group_max) grp.push_back(k);
        }
    }
    grp.push_back(dev->nranks);
    const int ngroups = (int)grp.size() - 1;
    // cell runs before the face reductions where a brick's slots are far
    // larger than L2 (the reductions then mostly go to DRAM)
    int l2 = 0;
    cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev->cuda_device);
    int runs = max_brick * sizeof(float4) > 8 * (size_t)l2 ? 1 : 0;
    if (const char* env = getenv("DPV_FACE_RUNS")) runs = atoi(env) != 0;
    if (faces && ngroups == 1) {
        cudaEvent_t tc = stage_start(dev);
        CK(cudaMemsetAsync(dev->d_gface, 0, dev->gface_slots * sizeof(float4), dev->stream), "zero face buffer");
        stage_stop(dev, DPV_STAGE_FACE, tc);
    } else if (dL_dvol && !faces) {
        // the scalar atomics add into the field; the face-buffer groups'
        // gathers store each node in the first group that reaches it
        CK(cudaMemsetAsync(dL_dvol, 0, sizeof(float) * (size_t)dev->dims[0] * dev->dims[1] * dev->dims[2], dev->stream),
           "zero dvol");
    }
    CK(cudaMemsetAsync(&dev->d_counters->samples_bwd, 0, sizeof(unsigned long long), dev->stream), "reset counter");
    cudaEvent_t t0 = stage_start(dev);
    CK(launch_composite_bwd(P, dev->d_tile_first, dev->d_tile_count, dev->d_frag_rgba, dev->d_frag_key,
                            (const float4*)dL_drgba, dev->d_frag_grad, dev->stream),
       "composite backward");
    stage_stop(dev, DPV_STAGE_COMPOSITE_BWD, t0);
    const bool persistent = (dev->frame.flags & DPV_FRAME_PERSISTENT) != 0;
    Schedule sch{dev->d_sched, dev->d_work, 0};   // the pull order built by the render
    if (!staged && faces) {
        // the replays are timed as DPV_STAGE_MARCH_BWD, the clears and
        // gathers of the face buffer as DPV_STAGE_FACE
        for (int g = 0; g < ngroups; ++g) {
            const FaceGroup fg{grp[g], grp[g + 1], (long long)dev->gface_off_h[grp[g]], runs};
            if (ngroups > 1) {
                cudaEvent_t tc = stage_start(dev);
                CK(cudaMemsetAsync(dev->d_gface, 0,
                                   (dev->gface_off_h[fg.k1] - dev->gface_off_h[fg.k0]) * sizeof(float4), dev->stream),
                   "zero face buffer");
                stage_stop(dev, DPV_STAGE_FACE, tc);
            }
            t0 = stage_start(dev);
            CK(launch_march_bwd(dev->bricks[0].dtype, dev->gather, P, dev->d_cams, dev->d_bricks, dev->d_scales,
                                dev->d_items, dev->n_items, dev->d_tf, dev->d_frag_rgba, dev->d_frag_key,
                                dev->d_frag_grad, dL_dtf, nullptr, dev->d_gface, dev->d_counters, dev->stream,
                                persistent ? &sch : nullptr, &fg),
               "march backward");
            stage_stop(dev, DPV_STAGE_MARCH_BWD, t0);
            t0 = stage_start(dev);
            CK(launch_face_gather(dev->d_bricks, dev->nranks, dev->d_nb_first, dev->d_nb, dev->max_rows,
                                  dev->d_gface, dev->dims, dL_dvol, dev->stream, ngroups > 1 ? &fg : nullptr),
               "face gather");
            stage_stop(dev, DPV_STAGE_FACE, t0);
        }
        dev->launches += ngroups * ((dev->n_items > 0 ? 1 : 0) + (dev->max_rows > 0 ? 1 : 0));
        return finish_backward(dev);
    }
    t0 = stage_start(dev);
    if (!staged) {
        CK(launch_march_bwd(dev->bricks[0].dtype, dev->gather, P, dev->d_cams, dev->d_bricks, dev->d_scales,
                            dev->d_items, dev->n_items, dev->d_tf, dev->d_frag_rgba, dev->d_frag_key,
                            dev->d_frag_grad, dL_dtf, dL_dvol, nullptr, dev->d_counters, dev->stream,
                            persistent ? &sch : nullptr),
           "march backward");
        dev->launches += dev->n_items > 0 ? 1 : 0;
    } else
        CK(launch_march_bwd_staged(dev->bricks[0].dtype, P, dev->d_cams, dev->d_bricks, dev->d_scales, dev->d_items,
                                   dev->n_items, dev->d_tf, dev->d_frag_rgba, dev->d_frag_key, dev->d_frag_grad,
                                   dL_dtf, dL_dvol, dev->d_counters, dev->stream),
           "march backward");
    stage_stop(dev, DPV_STAGE_MARCH_BWD, t0);
    if (staged) dev->launches += dev->n_items > 0 ? 1 : 0;
    return finish_backward(dev);
}

dpv_status dpvGetStats(dpv_device dev, dpv_stats* out) {
    dpv_status s = check_dev(dev);
    if (s) return s;
    if (!out) return fail(DPV_ERR_INVALID_ARG, "out NULL");
    memset(out, 0, sizeof *out);
    if (!dev->d_counters) return DPV_OK;
    DeviceGuard g(dev->cuda_device);
    Counters c;
    CK(cudaMemcpyAsync(&c, dev->d_counters, sizeof c, cudaMemcpyDeviceToHost, dev->stream), "read counters");
    CK(cudaStreamSynchronize(dev->stream), "read counters");
    out->samples_forward = c.samples_fwd;
    out->samples_backward = c.samples_bwd;
    out->work_items = (uint64_t)dev->n_items;
    out->fragment_bytes = (uint64_t)dev->frag_cap * dev->P.tp * (sizeof(float4) + sizeof(int) +
                                                                  (dev->d_frag_grad ? sizeof(float4) : 0));
    out->error_flags = c.err;
    out->max_fragments = c.max_frag;
    resolve_timers(dev);
    for (int i = 0; i < DPV_NUM_STAGES; ++i) {
        out->stage_ms[i] = dev->stage_ms[i];
        out->stage_calls[i] = dev->stage_calls[i];
    }
    out->kernel_launches = dev->launches;
    out->graph_launches = dev->graph_launches;
    out->samples_shadow = c.samples_shadow;
    return DPV_OK;
}

dpv_status dpvAutotune(dpv_device dev, int frames, dpv_tune_result* out) {
    dpv_status s = check_dev(dev);
    if (s) return s;
    if (frames < 1) return fail(DPV_ERR_INVALID_ARG, "frames must be >= 1");
    if (!dev->has_frame) return fail(DPV_ERR_STATE, "no frame parameters");
    DeviceGuard g(dev->cuda_device);
    const dpv_frame_desc keep = dev->frame;
    const int tune_bits =
        DPV_FRAME_LINEAR | DPV_FRAME_CELL | DPV_FRAME_QUAD | DPV_FRAME_PERSISTENT | DPV_FRAME_STAGED;
    const int tiles[4][2] = {{16, 16}, {32, 8}, {8, 32}, {64, 4}};
    // layouts: cell (where it fits), quad, linear; each per-item and persistent
    std::vector<int> sched_bits;
    const int layouts[3] = {DPV_FRAME_CELL, DPV_FRAME_QUAD, DPV_FRAME_LINEAR};
    const bool cell_ok = cell_fits(dev);
    for (int l : layouts) {
        if (l == DPV_FRAME_CELL && !cell_ok) continue;
        sched_bits.push_back(l);
        sched_bits.push_back(l | DPV_FRAME_PERSISTENT);
    }
    cudaEvent_t a = nullptr, b = nullptr;
    CK(cudaEventCreate(&a), "tune event");
    CK(cudaEventCreate(&b), "tune event");
    const bool prof = dev->profiling;
    dev->profiling = false;
    float best = 1e30f;
    dpv_frame_desc best_f = keep;
    int tried = 0;
    // layout outermost: each layout is built once
    for (int sb : sched_bits) {
        for (auto& t : tiles) {
            dpv_frame_desc f = keep;
            f.tile_w = t[0];
            f.tile_h = t[1];
            f.flags = (keep.flags & ~(tune_bits | DPV_FRAME_GRAPH)) | sb;
            dev->frame = f;
            dev->dirty = true;
            if ((s = dpvRenderFrame(dev)) != DPV_OK) break;
            CK(cudaEventRecord(a, dev->stream), "tune record");
            for (int i = 0; i < frames && s == DPV_OK; ++i) s = dpvRenderFrame(dev);
            if (s != DPV_OK) break;
            CK(cudaEventRecord(b, dev->stream), "tune record");
            CK(cudaEventSynchronize(b), "tune sync");
            float ms = 0.0f;
            CK(cudaEventElapsedTime(&ms, a, b), "tune time");
            ms /= frames;
            ++tried;
            if (ms < best) {
                best = ms;
                best_f = f;
            }
        }
        if (s != DPV_OK) break;
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    dev->profiling = prof;
    best_f.flags |= keep.flags & DPV_FRAME_GRAPH;
    dev->frame = best_f;
    dev->dirty = true;
    if (s != DPV_OK) {
        dev->frame = keep;
        return s;
    }
    if ((s = dpvRenderFrame(dev)) != DPV_OK) return s;
    if (out) {
        out->tile_w = best_f.tile_w;
        out->tile_h = best_f.tile_h;
        out->flags = best_f.flags & tune_bits;
        out->ms = best;
        out->candidates = tried;
    }
    return DPV_OK;
}

dpv_status dpvResetStats(dpv_device dev) {
    dpv_status s = check_dev(dev);
    if (s) return s;
    DeviceGuard g(dev->cuda_device);
    resolve_timers(dev);
    for (int i = 0; i < DPV_NUM_STAGES; ++i) {
        dev->stage_ms[i] = 0.0;
        dev->stage_calls[i] = 0;
    }
    dev->launches = 0;
    dev->graph_launches = 0;
    return DPV_OK;
}

dpv_status dpvSetProfiling(dpv_device dev, int enable) {
    dpv_status s = check_dev(dev);
    if (s) return s;
    dev->profiling = enable != 0;
    return DPV_OK;
}

dpv_status dpvRelease(dpv_device dev) {
    if (!dev) return DPV_OK;
    {
        DeviceGuard g(dev->cuda_device);
        if (!dev->poisoned && dev->stream) cudaStreamSynchronize(dev->stream);
        for (auto& b : dev->bricks) {
            dev_free(b.data);
            dev_free(b.gather);
            dev_free(b.mm);
        }
        dev_free(dev->d_empty);
        dev_free(dev->d_tfz);
        free_shadow(dev);
        free_schedule(dev);
        free_frags(dev);
        dev_free(dev->d_gface);
        dev_free(dev->d_nb_first);
        dev_free(dev->d_nb);
        dev_free(dev->d_scales);
        dev_free(dev->d_tmp);
        dev_free(dev->d_bricks);
        dev_free(dev->d_tf);
        dev_free(dev->d_cam_in);
        dev_free(dev->d_cams);
        dev_free(dev->d_camd);
        dev_free(dev->d_rays);
        dev_free(dev->d_out_rgba);
        dev_free(dev->d_out_depth);
        dev_free(dev->d_order);
        for (auto& m : dev->frag_maps) dev_free(m.second.ptr);
        dev->frag_maps.clear();
        dev_free(dev->d_counters);
        dev_free(dev->d_sched);
        dev_free(dev->d_hist);
        dev_free(dev->d_tmp64);
        free_graph(dev);
        if (dev->copy_stream) {
            cudaStreamSynchronize(dev->copy_stream);
            cudaStreamDestroy(dev->copy_stream);
        }
        for (int k = 0; k < 2; ++k) {
            dev_free(dev->d_stage_rgba[k]);
            dev_free(dev->d_stage_depth[k]);
            if (dev->ev_staged[k]) cudaEventDestroy(dev->ev_staged[k]);
            if (dev->ev_drained[k]) cudaEventDestroy(dev->ev_drained[k]);
        }
        if (dev->cap_stream) cudaStreamDestroy(dev->cap_stream);
        for (int k = 0; k < 2; ++k) {
            if (dev->ev_tf_stage[k]) {
                cudaEventSynchronize(dev->ev_tf_stage[k]);
                cudaEventDestroy(dev->ev_tf_stage[k]);
            }
            if (dev->h_tf_stage[k]) cudaFreeHost(dev->h_tf_stage[k]);
        }
        if (dev->ev_done) cudaEventDestroy(dev->ev_done);
        for (auto& t : dev->pending) {
            cudaEventDestroy(t.a);
            cudaEventDestroy(t.b);
        }
        for (auto e : dev->event_pool) cudaEventDestroy(e);
        cudaGetLastError();
    }
    delete dev;
    return DPV_OK;
}

}  // extern "C"
