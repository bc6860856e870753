// noalloc.cu -- dpvRenderNoAlloc: the render of dpvRenderFrame for one
// camera, as a single call that allocates no device memory.
//
// Who needs it: callers that may not call cudaMalloc themselves or have the
// library do so -- applications whose device memory is owned by their own
// pool or by a framework's caching allocator (a cudaMalloc behind its back
// can fail or fragment what it manages), and latency-bound render loops that
// cannot afford the device-wide synchronisation cudaMalloc and cudaFree
// imply.  The caller passes every
// input and output as device memory it already owns; the intermediate
// buffers (brick table, rays, work list, fragment pool) live in one
// file-scope device array of fixed size, kScratchBytes, which every GPU that
// loads this library holds until the process exits.
//
// The array is shared by all calls: calls that overlap on the GPU (on two
// streams, or from two host threads) race on it and must be serialised by
// the caller.  Each call re-initialises what must start cleared.
#include <string.h>

#include <mutex>
#include <string>
#include <vector>

#include "../../include/dpv.h"
#include "dpv_internal.cuh"
#include "launch.h"

using namespace dpv;

namespace {

constexpr size_t kScratchBytes = 64ull << 20;   // 64 MiB per GPU
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

std::mutex g_mu;
void* g_scratch_ptr[kMaxDevices] = {};

dpv_status na_fail(dpv_status s, const char* msg) {
    dpv::set_last_error(msg);
    return s;
}

// Device address of the scratch array on the current device, looked up on
// the first call on each device (with that device current) and cached; the
// host-side name of the array is only a host stand-in, not a device address.
dpv_status scratch_address(int device, unsigned char** out) {
    if (device < 0 || device >= kMaxDevices) return na_fail(DPV_ERR_UNSUPPORTED, "device index too large");
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_ptr[device]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess || !p) {
            std::string m = std::string("cudaGetSymbolAddress of the scratch array: ") + cudaGetErrorString(e);
            return na_fail(DPV_ERR_CUDA, m.c_str());
        }
        g_scratch_ptr[device] = p;
    }
    *out = (unsigned char*)g_scratch_ptr[device];
    return DPV_OK;
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// The call's small host tables (brick table, scales, camera) reach the
// device as kernel parameters, under 4 KB per launch, instead of copies
// from host memory: nothing reads the host memory behind them after the
// call returns, and nothing needs a staging buffer.
struct Words {
    unsigned n;
    unsigned w[1000];
};

__global__ void k_put_words(Words b, unsigned* dst) {
    for (unsigned i = threadIdx.x; i < b.n; i += blockDim.x) dst[i] = b.w[i];
}

cudaError_t put_words(void* dst, const void* src, size_t bytes, cudaStream_t st) {
    const unsigned* s = (const unsigned*)src;
    unsigned* d = (unsigned*)dst;
    size_t n = bytes / 4;
    Words b;
    for (size_t i = 0; i < n; i += 1000) {
        b.n = (unsigned)(n - i < 1000 ? n - i : 1000);
        memcpy(b.w, s + i, 4 * (size_t)b.n);
        k_put_words<<<1, 256, 0, st>>>(b, d + i);
    }
    return cudaGetLastError();
}

}  // namespace

extern "C" dpv_status dpvRenderNoAlloc(const dpv_noalloc_scene* sc, const dpv_camera* cam, const dpv_frame_desc* fr,
                                       float* rgba, float* depth, void* cuda_stream) {
    dpv::set_last_error("");
    if (!sc || !cam || !fr || !rgba || !depth) return na_fail(DPV_ERR_INVALID_ARG, "NULL argument");
    const int K = sc->num_ranks;
    if (K < 1 || K > MAX_RANKS || !sc->bricks) return na_fail(DPV_ERR_INVALID_ARG, "num_ranks must be 1..255");
    if ((int)sc->storage < 0 || (int)sc->storage > 3) return na_fail(DPV_ERR_INVALID_ARG, "bad storage dtype");
    if (!sc->tf_rgba || sc->tf_n < 2 || sc->tf_n > MAX_TF || !(sc->vmax > sc->vmin))
        return na_fail(DPV_ERR_INVALID_ARG, "bad transfer function");
    if (!(sc->spacing > 0.0f)) return na_fail(DPV_ERR_INVALID_ARG, "spacing must be > 0");
    for (int a = 0; a < 3; ++a)
        if (sc->dims[a] < 2) return na_fail(DPV_ERR_INVALID_ARG, "dims must be >= 2");
    if (fr->width < 1 || fr->height < 1 || !(fr->step_voxels > 0.0f) || !(fr->sigma_max >= 0.0f))
        return na_fail(DPV_ERR_INVALID_ARG, "bad frame parameters");
    int tw = fr->tile_w > 0 ? fr->tile_w : 16, th = fr->tile_h > 0 ? fr->tile_h : 16;
    if (tw % 8 || th % 4 || tw * th > 256) return na_fail(DPV_ERR_INVALID_ARG, "bad tile size");
    if (((uintptr_t)rgba & 15) || ((uintptr_t)depth & 3)) return na_fail(DPV_ERR_INVALID_ARG, "misaligned output");
    // the march reads the table as float4
    if ((uintptr_t)sc->tf_rgba & 15)
        return na_fail(DPV_ERR_INVALID_ARG, "transfer function not 16-byte aligned");
    if (const char* why = camera_problem(*cam)) {
        std::string m = std::string("camera: ") + why;
        return na_fail(DPV_ERR_INVALID_ARG, m.c_str());
    }
    if (fr->flags & (DPV_FRAME_ISO | DPV_FRAME_ORDERED | DPV_FRAME_SKIP | DPV_FRAME_DEEP | DPV_FRAME_SHADOW |
                     DPV_FRAME_ORDER))
        return na_fail(DPV_ERR_UNSUPPORTED,
                       "iso-surface, ordered, skipping, deep and shadowed frames and the order image need "
                       "dpvRenderFrame");

    // bricks: owned ranges must tile the volume exactly
    std::vector<BrickDev> table(K);
    std::vector<float> scales(K);
    long long total = 0;
    for (int k = 0; k < K; ++k) {
        const dpv_noalloc_brick& h = sc->bricks[k];
        if (!h.data) return na_fail(DPV_ERR_INVALID_ARG, "brick data is NULL");
        BrickDev& b = table[k];
        long long v = 1, nodes = 1;
        for (int a = 0; a < 3; ++a) {
            if (h.owned_lo[a] < 0 || h.owned_hi[a] > sc->dims[a] || h.owned_lo[a] >= h.owned_hi[a])
                return na_fail(DPV_ERR_INVALID_ARG, "owned range outside the volume or empty");
            v *= (long long)(h.owned_hi[a] - h.owned_lo[a]);
            b.s_lo[a] = h.owned_lo[a] - 1 < 0 ? 0 : h.owned_lo[a] - 1;
            int s_hi = h.owned_hi[a] > sc->dims[a] - 1 ? sc->dims[a] - 1 : h.owned_hi[a];
            b.s_n[a] = s_hi - b.s_lo[a] + 1;
            nodes *= b.s_n[a];
            float lo = (float)h.owned_lo[a] - 0.5f, hi = (float)h.owned_hi[a] - 0.5f;
            b.r0[a] = lo < 0.0f ? 0.0f : lo;
            b.r1[a] = hi > (float)(sc->dims[a] - 1) ? (float)(sc->dims[a] - 1) : hi;
            b.closed[a] = h.owned_hi[a] >= sc->dims[a] ? 1 : 0;
            b.o_lo[a] = h.owned_lo[a];
            b.o_hi[a] = h.owned_hi[a];
        }
        b.gface_off = 0;   // no backward here
        if (nodes > 0x7fffffffLL) return na_fail(DPV_ERR_UNSUPPORTED, "brick too large");
        total += v;
        for (int m = 0; m < k; ++m) {
            const dpv_noalloc_brick& c = sc->bricks[m];
            bool overlap = true;
            for (int a = 0; a < 3; ++a)
                overlap = overlap && h.owned_lo[a] < c.owned_hi[a] && c.owned_lo[a] < h.owned_hi[a];
            if (overlap) return na_fail(DPV_ERR_INVALID_ARG, "owned ranges overlap");
        }
        b.data = h.data;
        b.sx = b.s_n[0];
        b.sxy = b.s_n[0] * b.s_n[1];
        b.scale_idx = k;
        b.pad = 0;
        scales[k] = h.scale > 0.0f ? h.scale : 1.0f;
    }
    if (total != (long long)sc->dims[0] * sc->dims[1] * sc->dims[2])
        return na_fail(DPV_ERR_INVALID_ARG, "owned ranges do not cover the volume exactly");

    FrameParams P{};
    P.W = fr->width;
    P.H = fr->height;
    P.tw = tw;
    P.th = th;
    P.ntx = (P.W + tw - 1) / tw;
    P.nty = (P.H + th - 1) / th;
    P.ncam = 1;
    P.tp = tw * th;
    P.dt = fr->step_voxels * sc->spacing;
    P.inv_dt = 1.0f / P.dt;
    P.sigma_max = fr->sigma_max;
    P.ert = fr->ert_threshold;
    P.ert_on = (fr->ert_threshold > 0.0f && fr->ert_threshold < 1.0f) ? 1 : 0;
    P.vmin = sc->vmin;
    P.vmax = sc->vmax;
    P.tf_scale = (float)(sc->tf_n - 1) / (sc->vmax - sc->vmin);
    P.tf_bias = -P.vmin * P.tf_scale;
    P.sdt = P.sigma_max * P.dt;
    P.ntf = sc->tf_n;
    for (int a = 0; a < 3; ++a) P.dims[a] = sc->dims[a];
    P.nbricks = K;
    P.order_stride = 0;
    P.deep = 1;

    // carve the scratch array: worst-case work list (every tile sees every
    // brick), so no count has to be read back
    const size_t ntiles = (size_t)P.ntx * P.nty;
    const size_t cap = ntiles * K;
    const size_t npix = (size_t)P.W * P.H;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o = off;
        off = align256(off + bytes);
        return o;
    };
    size_t o_table = take(sizeof(BrickDev) * K);
    size_t o_scales = take(sizeof(float) * K);
    size_t o_camin = take(sizeof(CamIn));
    size_t o_cam = take(sizeof(CamBasis));
    size_t o_camd = take(sizeof(CamBasisDF));
    size_t o_counters = take(sizeof(Counters));
    size_t o_rays = take(RAY_VECS * sizeof(float4) * npix);
    size_t o_rects = take(sizeof(int4) * K);
    size_t o_count = take(sizeof(int) * ntiles);
    size_t o_first = take(sizeof(int) * ntiles);
    size_t o_items = take(sizeof(Item) * cap);
    size_t o_frgba = take(sizeof(float4) * cap * P.tp);
    size_t o_fkey = take(sizeof(int) * cap * P.tp);
    if (off > kScratchBytes || cap * P.tp > 0x7fffffffULL) {
        char buf[256];
        snprintf(buf, sizeof buf,
                 "frame needs %zu bytes of scratch; the allocation-free render holds %zu (reduce width x height "
                 "or ranks, or use dpvRenderFrame)",
                 off, kScratchBytes);
        return na_fail(DPV_ERR_INVALID_ARG, buf);
    }
    P.items_cap = (int)cap;

    int device = 0;
    cudaError_t e = cudaGetDevice(&device);
    if (e != cudaSuccess) return na_fail(DPV_ERR_CUDA, cudaGetErrorString(e));
    unsigned char* base = nullptr;
    dpv_status s = scratch_address(device, &base);
    if (s) return s;
    cudaStream_t st = (cudaStream_t)cuda_stream;

    BrickDev* d_table = (BrickDev*)(base + o_table);
    float* d_scales = (float*)(base + o_scales);
    CamIn* d_camin = (CamIn*)(base + o_camin);
    CamBasis* d_cam = (CamBasis*)(base + o_cam);
    CamBasisDF* d_camd = (CamBasisDF*)(base + o_camd);
    Counters* d_counters = (Counters*)(base + o_counters);
    float4* d_rays = (float4*)(base + o_rays);
    int4* d_rects = (int4*)(base + o_rects);
    int* d_count = (int*)(base + o_count);
    int* d_first = (int*)(base + o_first);
    Item* d_items = (Item*)(base + o_items);
    float4* d_frgba = (float4*)(base + o_frgba);
    int* d_fkey = (int*)(base + o_fkey);
    P.rays = d_rays;

    CamIn ci;
    memcpy(&ci, cam, sizeof ci);
#define NA_CK(x)                                                         \
    do {                                                                 \
        cudaError_t e_ = (x);                                            \
        if (e_ != cudaSuccess) return na_fail(DPV_ERR_CUDA, cudaGetErrorString(e_)); \
    } while (0)
    static_assert(sizeof(BrickDev) % 4 == 0 && sizeof(CamIn) % 4 == 0, "tables travel as 32-bit words");
    NA_CK(put_words(d_table, table.data(), sizeof(BrickDev) * K, st));
    NA_CK(put_words(d_scales, scales.data(), sizeof(float) * K, st));
    NA_CK(put_words(d_camin, &ci, sizeof ci, st));
    // the array keeps the previous call's contents: clear the counters and
    // mark every work-list entry invalid before the cull fills it
    NA_CK(cudaMemsetAsync(d_counters, 0, sizeof(Counters), st));
    NA_CK(cudaMemsetAsync(d_items, 0xFF, sizeof(Item) * cap, st));
    float3 og = make_float3(sc->origin[0], sc->origin[1], sc->origin[2]);
    NA_CK(launch_cull(P, d_camin, og, sc->spacing, d_cam, d_camd, d_rays, d_table, d_rects, d_count, d_first, d_items,
                      (int)cap, d_counters, true, st));
    NA_CK(launch_march_fwd((int)sc->storage, GATHER_LINEAR, P, d_cam, d_table, d_scales, d_items, (int)cap,
                           (const float4*)sc->tf_rgba, d_frgba, d_fkey, d_counters, st));
    NA_CK(launch_composite_fwd(P, 1.0f / sc->spacing, d_cam, d_first, d_count, d_items, d_frgba, d_fkey,
                               (float4*)rgba, depth, nullptr, st));
#undef NA_CK
    (void)npix;
    return DPV_OK;
}
