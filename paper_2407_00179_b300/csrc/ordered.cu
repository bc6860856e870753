// ordered.cu -- the visibility-ordered march with global early termination
// (DPV_FRAME_ORDERED, sm_103a).
//
// Each ray marches the bricks it crosses in its own front-to-back order,
// carrying colour and transmittance from brick to brick, and stops once the
// accumulated opacity passes the threshold: the fixed-order, occlusion-aware
// relative of sort-last compositing (IceT-style, §5.1.1, §8.2).  The per-sample
// arithmetic is the sort-last march's (dpv_internal.cuh), bit for bit.
#include "dpv_internal.cuh"
#include "launch.h"

#include <algorithm>

namespace dpv {

// ===========================================================================
// visibility-ordered march with global early termination (DPV_FRAME_ORDERED)
// ===========================================================================
//
// One thread per pixel.  Each thread finds where its ray enters every brick
// the tile's work list names (the first sample index of the brick's
// segment), takes the segments front to back, and marches them in that
// order from each brick's own storage (ghost layer included), carrying the
// accumulated colour and transmittance from brick to brick; once the
// accumulated opacity passes the threshold no further sample, in this brick
// or behind it, is evaluated.  The frame is written directly.  Two launch
// forms: one CTA per (camera, tile), or a persistent grid whose warps pull
// 32 pixels at a time (DPV_FRAME_PERSISTENT); the same frame bit for bit.

// The samples of one brick segment, continuing (C, Tr); true once the
// accumulated opacity passed the early-termination threshold.  Adds the
// samples it evaluated to nsamp.
template <typename T, int GL, bool SKIP>
__device__ __forceinline__ bool march_segment(const FrameParams& P, const BrickDev& b, float scale,
                                              const float4* s_tf, const MarchState& m, float& C0, float& C1,
                                              float& C2, float& Tr, unsigned long long& nsamp) {
    const int n = m.j1 - m.j0;
    SampleWalker wk;
    wk.init(b);
    if ((GL == GATHER_CELL || GL == GATHER_QUAD) && !SKIP) {
        // the next sample's cell (or faces) in flight during this sample's
        // arithmetic and the TF entries kept across an interval, as in the
        // sort-last march (interpolation and lookup bit-identical)
        GatherRaw<T, GL == GATHER_CELL ? GATHER_CELL : GATHER_QUAD> raw;
        TFCache<GL == GATHER_QUAD> tfc;
        int ix, iy, iz;
        float fx, fy, fz;
        wk.at(m, 0, ix, iy, iz, fx, fy, fz);
        raw.fetch(b, ix, iy, iz);
        int k = 0;
        bool stop = false;
        auto shade = [&](const float v[8], float cx, float cy, float cz) {
            float s = lerp_cell<T>(v, cx, cy, cz, scale);
            const float4 c = tfc.lookup(s_tf, P, s);
            float al = sample_alpha(P, c.w);
            float ta = Tr * al;
            C0 = fmaf(ta, c.x, C0);
            C1 = fmaf(ta, c.y, C1);
            C2 = fmaf(ta, c.z, C2);
            Tr = Tr - ta;
            return P.ert_on && 1.0f - Tr > P.ert;
        };
        // the last sample after the loop, which then tests no bound for
        // the look-ahead (as in the sort-last march)
        for (; k + 1 < n; ++k) {
            float v[8];
            raw.decode(v);
            const float cx = fx, cy = fy, cz = fz;
            wk.template at<!(GL == GATHER_CELL && sizeof(T) == 4)>(m, k + 1, ix, iy, iz, fx, fy, fz);
            raw.fetch(b, ix, iy, iz);
            if (shade(v, cx, cy, cz)) {
                ++k;
                stop = true;
                break;
            }
        }
        if (!stop && n > 0) {
            float v[8];
            raw.decode(v);
            stop = shade(v, fx, fy, fz);
            ++k;
        }
        nsamp += (unsigned)k;
        return stop;
    }
    const T* data = (const T*)b.data;
    CornerCache<T, GL> cc;
    int mlast = -1;
    bool mempty = false;
    for (int k = 0; k < n; ++k) {
        int ix, iy, iz;
        float fx, fy, fz;
        wk.at(m, k, ix, iy, iz, fx, fy, fz);
        if (SKIP) {
            const int mi = (iz >> MACRO_SHIFT) * b.mxy + (iy >> MACRO_SHIFT) * b.mx + (ix >> MACRO_SHIFT);
            if (mi != mlast) {
                mlast = mi;
                mempty = b.empty[mi] != 0;
            }
            if (mempty) {
                k = macro_last(m, wk, k, n, ix, iy, iz);
                continue;
            }
        }
        float s = trilinear<T, GL>(b, data, scale, cc, ix, iy, iz, fx, fy, fz);
        TFSample c = tf_lookup(s_tf, P, s);
        float al = sample_alpha(P, c.v.w);
        float ta = Tr * al;
        C0 = fmaf(ta, c.v.x, C0);
        C1 = fmaf(ta, c.v.y, C1);
        C2 = fmaf(ta, c.v.z, C2);
        Tr = Tr - ta;
        ++nsamp;
        if (P.ert_on && 1.0f - Tr > P.ert) return true;
    }
    return false;
}

// The work-list slot of the ray's segment with the smallest first sample
// index above `last` (-1: none), and that index, scanning the list.
// Only the ray's slab intersection with each candidate brick is needed
// (the pixel's ray is loaded once per call, not kept live across the
// march); the sample anchor of brick_samples is computed for the chosen
// segment alone.
__device__ __forceinline__ int next_segment(const FrameParams& P, const CamBasis& cam, int c, const BrickDev* bricks,
                                            const Item* items, long long first, int cnt, int px, int py, int last,
                                            int& j0) {
    Ray r;
    load_ray(cam, P, c, px, py, r);
    int best = KEY_EMPTY, bs = -1;
    for (int q = 0; q < cnt; ++q) {
        const Item it = items[first + q];
        if (!item_ok(it, P)) continue;
        int a, e;
        if (!segment_range(P, r, bricks[it.brick], a, e)) continue;
        if (a > last && a < best) {
            best = a;
            bs = q;
        }
    }
    j0 = best;
    return bs;
}

// Tile lists of at most this many items keep each ray's segment entries in
// shared memory, one column per thread: the list is scanned once per ray
// instead of once per segment.
constexpr int ORD_CACHE = 16;

// The pixel (px, py) of camera c, whose tile's work list is `ct`: its ray
// marched through its brick segments front to back; writes the pixel (and
// its order-map row).  s_entry is this thread's column of the entry cache
// (stride `col`).  Returns the samples evaluated.
template <typename T, int GL, bool SKIP>
__device__ __forceinline__ unsigned long long ordered_ray(const FrameParams& P, const CamBasis* cams,
                                                          const BrickDev* bricks, const float* scales,
                                                          const int* tile_first, const int* tile_count,
                                                          const Item* items, const float4* s_tf, int* s_entry,
                                                          int col, int c, int ct, int px, int py, float4* out_rgba,
                                                          float* out_depth, unsigned char* order) {
    unsigned long long nsamp = 0;
    long long first = tile_first[ct];
    int cnt = tile_count[ct];
    if (first < 0 || first + cnt > P.items_cap) cnt = 0;    // list overflowed: error bit already set
    const CamBasis cam = cams[c];
    const long long pix = ((long long)c * P.H + py) * P.W + px;
    unsigned char* ord = order ? order + pix * P.order_stride : nullptr;
    float C0 = 0.f, C1 = 0.f, C2 = 0.f, Tr = 1.0f;
    int depth_key = KEY_EMPTY, last = -1, i = 0;
    bool stop = false;
    const bool cached = cnt <= ORD_CACHE;
    if (cached) {
        Ray r;
        load_ray(cam, P, c, px, py, r);
        for (int q = 0; q < cnt; ++q) {
            const Item it = items[first + q];
            int a = KEY_EMPTY, e;
            if (!item_ok(it, P) || !segment_range(P, r, bricks[it.brick], a, e)) a = KEY_EMPTY;
            s_entry[q * col] = a;
        }
    }
    // the ray's brick segments front to back: each step selects the
    // segment with the smallest first sample index after the last one
    for (;; ++i) {
        int j0, q;
        if (cached) {
            j0 = KEY_EMPTY;
            q = -1;
            for (int u = 0; u < cnt; ++u) {
                const int a = s_entry[u * col];
                if (a > last && a < j0) {
                    j0 = a;
                    q = u;
                }
            }
        } else {
            q = next_segment(P, cam, c, bricks, items, first, cnt, px, py, last, j0);
        }
        if (q < 0) break;
        last = j0;
        const Item it = items[first + q];
        if (ord && i < P.order_stride) ord[i] = (unsigned char)it.brick;
        if (stop) continue;                    // behind the termination: listed, not marched
        const BrickDev b = bricks[it.brick];
        MarchState m;
        if (!brick_samples(P, cam, c, b, px, py, m)) continue;
        const float Tb = Tr;
        stop = march_segment<T, GL, SKIP>(P, b, scales[b.scale_idx], s_tf, m, C0, C1, C2, Tr, nsamp);
        if (Tr < Tb && depth_key == KEY_EMPTY) depth_key = m.j0;
        if (stop && !ord) break;
    }
    if (ord)
        for (; i < P.order_stride; ++i) ord[i] = 0xFF;
    out_rgba[pix] = make_float4(C0, C1, C2, 1.0f - Tr);
    float depth = __int_as_float(0x7f800000);
    if (depth_key != KEY_EMPTY) {
        Ray r;
        load_ray(cam, P, c, px, py, r);
        depth = r.te + ((float)depth_key + 0.5f) * P.dt;
    }
    out_depth[pix] = depth;
    return nsamp;
}

// 4 CTAs per SM (64 registers) for the pipelined cell- and quad-layout
// marches, 5 (48 registers) for the others
template <int GL, bool SKIP>
constexpr int ordered_min_ctas() {
    return ((GL == GATHER_CELL || GL == GATHER_QUAD) && !SKIP) ? 4 : 5;
}

// The TF table, then the entry cache (ORD_CACHE ints per thread).
__device__ __forceinline__ int* stage_tf(const FrameParams& P, const float4* tf, float4* s_tf) {
    for (int i = threadIdx.x; i < P.ntf; i += blockDim.x) s_tf[i] = tf[i];
    __syncthreads();
    return reinterpret_cast<int*>(s_tf + P.ntf) + threadIdx.x;
}

template <typename T, int GL, bool SKIP>
__global__ void __launch_bounds__(256, ordered_min_ctas<GL, SKIP>())
    k_march_ordered(FrameParams P, const CamBasis* cams, const BrickDev* bricks, const float* scales,
                    const int* tile_first, const int* tile_count, const Item* items, const float4* tf,
                    float4* out_rgba, float* out_depth, unsigned char* order, Counters* counters) {
    extern __shared__ float4 s_tf[];
    int* s_entry = stage_tf(P, tf, s_tf);
    const int ct = blockIdx.x;
    const int ntiles = P.ntx * P.nty;
    const int c = ct / ntiles, tile = ct % ntiles;
    int lx, ly;
    tile_pixel(threadIdx.x, P.tw, lx, ly);
    const int px = (tile % P.ntx) * P.tw + lx, py = (tile / P.ntx) * P.th + ly;
    unsigned long long nsamp = 0;
    if (px < P.W && py < P.H)
        nsamp = ordered_ray<T, GL, SKIP>(P, cams, bricks, scales, tile_first, tile_count, items, s_tf, s_entry,
                                         blockDim.x, c, ct, px, py, out_rgba, out_depth, order);
    nsamp = warp_sum_u64(nsamp);
    if ((threadIdx.x & 31) == 0 && nsamp) atomicAdd(&counters->samples_fwd, nsamp);
}

// Persistent form: a grid sized to the GPU whose warps each pull one warp's
// share of a tile (32 pixels) at a time from a counter, so a warp whose rays
// terminate early takes the next pixels at once instead of waiting for the
// other warps of its tile, and no CTA waits for its slowest warp.
template <typename T, int GL, bool SKIP>
__global__ void __launch_bounds__(256, ordered_min_ctas<GL, SKIP>())
    k_march_ordered_persistent(FrameParams P, const CamBasis* cams, const BrickDev* bricks, const float* scales,
                               const int* tile_first, const int* tile_count, const Item* items, const float4* tf,
                               float4* out_rgba, float* out_depth, unsigned char* order, Counters* counters,
                               unsigned int* work) {
    extern __shared__ float4 s_tf[];
    int* s_entry = stage_tf(P, tf, s_tf);
    const int lane = threadIdx.x & 31;
    const int ntiles = P.ntx * P.nty;
    const unsigned wpt = (unsigned)(P.tp >> 5);              // warps per tile
    const unsigned n_units = (unsigned)(P.ncam * ntiles) * wpt;
    unsigned long long nsamp = 0;
    for (;;) {
        __syncwarp();
        unsigned u = 0;
        if (lane == 0) u = atomicAdd(work, 1u);
        u = __shfl_sync(0xffffffffu, u, 0);
        if (u >= n_units) break;
        const int ct = (int)(u / wpt);
        const int c = ct / ntiles, tile = ct % ntiles;
        int lx, ly;
        tile_pixel((int)((u % wpt) * 32) + lane, P.tw, lx, ly);
        const int px = (tile % P.ntx) * P.tw + lx, py = (tile / P.ntx) * P.th + ly;
        if (px < P.W && py < P.H)
            nsamp += ordered_ray<T, GL, SKIP>(P, cams, bricks, scales, tile_first, tile_count, items, s_tf, s_entry,
                                              blockDim.x, c, ct, px, py, out_rgba, out_depth, order);
    }
    nsamp = warp_sum_u64(nsamp);
    if (lane == 0 && nsamp) atomicAdd(&counters->samples_fwd, nsamp);
}

template <typename T, int GL, bool SKIP>
static void ordered_launch_s(const FrameParams& P, const CamBasis* cams, const BrickDev* bricks, const float* scales,
                             const int* tile_first, const int* tile_count, const Item* items, const float4* tf,
                             float4* out_rgba, float* out_depth, unsigned char* order, Counters* counters,
                             unsigned int* work, cudaStream_t st) {
    const size_t smem = sizeof(float4) * P.ntf + sizeof(int) * ORD_CACHE * P.tp;
    const int nct = P.ncam * P.ntx * P.nty;
    if (work) {
        auto kern = k_march_ordered_persistent<T, GL, SKIP>;
        if (smem > 48 * 1024) cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        int per_sm = 0, dev = 0, nsm = 148;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, P.tp, smem);
        const int grid = std::min(nsm * std::max(per_sm, 1), nct);   // a CTA's warps take at least one tile
        cudaMemsetAsync(work, 0, sizeof(unsigned int), st);
        kern<<<grid, P.tp, smem, st>>>(P, cams, bricks, scales, tile_first, tile_count, items, tf, out_rgba,
                                       out_depth, order, counters, work);
        return;
    }
    if (smem > 48 * 1024)
        cudaFuncSetAttribute(k_march_ordered<T, GL, SKIP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_march_ordered<T, GL, SKIP><<<nct, P.tp, smem, st>>>(P, cams, bricks, scales, tile_first, tile_count, items, tf,
                                                          out_rgba, out_depth, order, counters);
}

template <typename T, int GL>
static void ordered_launch(const FrameParams& P, const CamBasis* cams, const BrickDev* bricks, const float* scales,
                           const int* tile_first, const int* tile_count, const Item* items, const float4* tf,
                           float4* out_rgba, float* out_depth, unsigned char* order, Counters* counters,
                           unsigned int* work, cudaStream_t st) {
    if (P.skip_on)
        ordered_launch_s<T, GL, true>(P, cams, bricks, scales, tile_first, tile_count, items, tf, out_rgba, out_depth,
                                      order, counters, work, st);
    else
        ordered_launch_s<T, GL, false>(P, cams, bricks, scales, tile_first, tile_count, items, tf, out_rgba,
                                       out_depth, order, counters, work, st);
}

cudaError_t launch_march_ordered(int dtype, int gather, const FrameParams& P, const CamBasis* cams,
                                 const BrickDev* bricks, const float* scales, const int* tile_first,
                                 const int* tile_count, const Item* items, const float4* tf, float4* out_rgba,
                                 float* out_depth, unsigned char* order, Counters* counters, unsigned int* work,
                                 cudaStream_t st) {
#define ORD(T)                                                                                                  \
    (gather == GATHER_CELL   ? ordered_launch<T, GATHER_CELL>(P, cams, bricks, scales, tile_first, tile_count,  \
                                                              items, tf, out_rgba, out_depth, order, counters, work, st) \
     : gather == GATHER_QUAD ? ordered_launch<T, GATHER_QUAD>(P, cams, bricks, scales, tile_first, tile_count,  \
                                                              items, tf, out_rgba, out_depth, order, counters, work, st) \
                             : ordered_launch<T, GATHER_LINEAR>(P, cams, bricks, scales, tile_first, tile_count, \
                                                                items, tf, out_rgba, out_depth, order, counters, work, st))
    switch (dtype) {
        case 0: ORD(float); break;
        case 1: ORD(__half); break;
        case 2: ORD(__nv_bfloat16); break;
        default: ORD(__nv_fp8_e4m3); break;
    }
#undef ORD
    return cudaGetLastError();
}

}  // namespace dpv
