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
// One CTA per (camera, tile).  Each thread finds where its ray enters every
// brick the tile's work list names (the first sample index of the brick's
// segment), sorts the segments front to back, and marches them in that
// order from each brick's own storage (ghost layer included), carrying the
// accumulated colour and transmittance from brick to brick; once the
// accumulated opacity passes the threshold no further sample, in this brick
// or behind it, is evaluated.  The frame is written directly.

// The samples of one brick segment, continuing (C, Tr); true once the
// accumulated opacity passed the early-termination threshold.
template <typename T, int GL, bool SKIP>
__device__ __forceinline__ bool march_segment(const FrameParams& P, const BrickDev& b, float scale,
                                              const float4* s_tf, const MarchState& m, float& C0, float& C1,
                                              float& C2, float& Tr, unsigned long long& nsamp) {
    const T* data = (const T*)b.data;
    const int n = m.j1 - m.j0;
    CornerCache<T, GL> cc;
    SampleWalker wk;
    wk.init(b);
    int mlast = -1;
    bool mempty = false;
    if (GL == GATHER_CELL && !SKIP) {
        // the next sample's cell in flight during this sample's arithmetic
        // (as in the sort-last march; interpolation bit-identical)
        CellRaw<T> raw;
        int ix, iy, iz;
        float fx, fy, fz;
        wk.at(m, 0, ix, iy, iz, fx, fy, fz);
        raw.fetch(b.gather, cell_slot(b, ix, iy, iz));
        for (int k = 0; k < n; ++k) {
            float v[8];
            raw.decode(v);
            const float cx = fx, cy = fy, cz = fz;
            if (k + 1 < n) {
                wk.at(m, k + 1, ix, iy, iz, fx, fy, fz);
                raw.fetch(b.gather, cell_slot(b, ix, iy, iz));
            }
            float s = lerp_cell<T>(v, cx, cy, cz, scale);
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
// index above `last` (-1: none), and that index.
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

// 4 CTAs per SM (64 registers) for the pipelined cell-layout march, 5 (48
// registers) for the others: measured best for each
template <int GL, bool SKIP>
constexpr int ordered_min_ctas() {
    return (GL == GATHER_CELL && !SKIP) ? 4 : 5;
}

template <typename T, int GL, bool SKIP>
__global__ void __launch_bounds__(256, ordered_min_ctas<GL, SKIP>()) k_march_ordered(FrameParams P, const CamBasis* cams,
                                                          const BrickDev* bricks, const float* scales,
                                                          const int* tile_first, const int* tile_count,
                                                          const Item* items, const float4* tf, float4* out_rgba,
                                                          float* out_depth, unsigned char* order,
                                                          Counters* counters) {
    extern __shared__ float4 s_tf[];
    for (int i = threadIdx.x; i < P.ntf; i += blockDim.x) s_tf[i] = tf[i];
    __syncthreads();
    const int ct = blockIdx.x;
    const int ntiles = P.ntx * P.nty;
    const int c = ct / ntiles, tile = ct % ntiles;
    int lx, ly;
    tile_pixel(threadIdx.x, P.tw, lx, ly);
    const int px = (tile % P.ntx) * P.tw + lx, py = (tile / P.ntx) * P.th + ly;
    unsigned long long nsamp = 0;
    if (px < P.W && py < P.H) {
        long long first = tile_first[ct];
        int cnt = tile_count[ct];
        if (first < 0 || first + cnt > P.items_cap) cnt = 0;    // list overflowed: error bit already set
        const CamBasis cam = cams[c];
        const long long pix = ((long long)c * P.H + py) * P.W + px;
        unsigned char* ord = order ? order + pix * P.order_stride : nullptr;
        float C0 = 0.f, C1 = 0.f, C2 = 0.f, Tr = 1.0f;
        int depth_key = KEY_EMPTY, last = -1, i = 0;
        bool stop = false;
        // the ray's brick segments front to back: each step selects the
        // segment with the smallest first sample index after the last one
        for (;; ++i) {
            int j0;
            const int q = next_segment(P, cam, c, bricks, items, first, cnt, px, py, last, j0);
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
    }
    nsamp = warp_sum_u64(nsamp);
    if ((threadIdx.x & 31) == 0 && nsamp) atomicAdd(&counters->samples_fwd, nsamp);
}

// ---------------------------------------------------------------------------
// persistent form with ray refill (DPV_FRAME_ORDERED | DPV_FRAME_PERSISTENT)
// ---------------------------------------------------------------------------
//
// In the per-tile form a warp runs until its longest ray has terminated;
// lanes whose rays stopped early idle meanwhile.  Here a grid sized to the
// GPU keeps every lane busy: a warp pulls 32 pixels (one warp's share of a
// tile) at a time from a counter, and a lane whose ray is finished takes the
// next pixel of the warp's share as soon as enough lanes of the warp are
// free.  A lane marches its open brick segment until the segment ends, the
// ray terminates, or REFILL_AT lanes have left the march since it started;
// it then leaves the march with its position saved (sample index, colour,
// transmittance) and resumes after the warp has refilled its free lanes and
// chosen the next segments of the lanes that need one.  The samples, their
// order along each ray and their arithmetic are the per-tile form's, so the
// frame is the same bit for bit.
constexpr int REFILL_AT = 8;

// Samples k.. of the ray's open segment in brick b, continuing (C, Tr).
// Returns 1 when the segment is done, 2 when the accumulated opacity passed
// the termination threshold, 0 when the lane left the march with k the next
// sample (fewer than `keep` lanes still marching).
template <typename T, int GL, bool SKIP>
__device__ __forceinline__ int march_resume(const FrameParams& P, const BrickDev& b, float scale,
                                            const float4* s_tf, const MarchState& m, int keep, int& k, float& C0,
                                            float& C1, float& C2, float& Tr, unsigned long long& nsamp) {
    const int n = m.j1 - m.j0;
    if (k >= n) return 1;
    SampleWalker wk;
    wk.init(b);
    if ((GL == GATHER_CELL || GL == GATHER_QUAD) && !SKIP) {
        // the next sample's cell (or faces) in flight during this sample's
        // arithmetic, as in the sort-last march
        GatherRaw<T, GL == GATHER_CELL ? GATHER_CELL : GATHER_QUAD> raw;
        int ix, iy, iz;
        float fx, fy, fz;
        wk.at(m, k, ix, iy, iz, fx, fy, fz);
        raw.fetch(b, ix, iy, iz);
        for (;;) {
            float v[8];
            raw.decode(v);
            const float cx = fx, cy = fy, cz = fz;
            const bool more = k + 1 < n;
            const bool leave = more && __popc(__activemask()) < keep;
            if (more && !leave) {
                wk.at(m, k + 1, ix, iy, iz, fx, fy, fz);
                raw.fetch(b, ix, iy, iz);
            }
            float s = lerp_cell<T>(v, cx, cy, cz, scale);
            TFSample c = tf_lookup(s_tf, P, s);
            float al = sample_alpha(P, c.v.w);
            float ta = Tr * al;
            C0 = fmaf(ta, c.v.x, C0);
            C1 = fmaf(ta, c.v.y, C1);
            C2 = fmaf(ta, c.v.z, C2);
            Tr = Tr - ta;
            ++k;
            ++nsamp;
            if (P.ert_on && 1.0f - Tr > P.ert) return 2;
            if (!more) return 1;
            if (leave) return 0;
        }
    }
    const T* data = (const T*)b.data;
    CornerCache<T, GL> cc;
    int mlast = -1;
    bool mempty = false;
    while (k < n) {
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
                k = macro_last(m, wk, k, n, ix, iy, iz) + 1;
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
        ++k;
        ++nsamp;
        if (P.ert_on && 1.0f - Tr > P.ert) return 2;
        if (k < n && __popc(__activemask()) < keep) return 0;
    }
    return 1;
}

// The ray's pixel: colour and opacity, and the depth of its first sample
// that changed the transmittance (infinity when none did).
__device__ __forceinline__ void write_pixel(const FrameParams& P, const CamBasis& cam, int c, int px, int py,
                                            float C0, float C1, float C2, float Tr, int depth_key, float4* out_rgba,
                                            float* out_depth) {
    const long long pix = ((long long)c * P.H + py) * P.W + px;
    out_rgba[pix] = make_float4(C0, C1, C2, 1.0f - Tr);
    float depth = __int_as_float(0x7f800000);
    if (depth_key != KEY_EMPTY) {
        Ray r;
        load_ray(cam, P, c, px, py, r);
        depth = r.te + ((float)depth_key + 0.5f) * P.dt;
    }
    out_depth[pix] = depth;
}

// 64 registers (4 CTAs per SM): the ray and segment state stay in
// registers across the refills
template <typename T, int GL, bool SKIP>
__global__ void __launch_bounds__(256, 4)
    k_march_ordered_refill(FrameParams P, const CamBasis* cams, const BrickDev* bricks, const float* scales,
                           const int* tile_first, const int* tile_count, const Item* items, const float4* tf,
                           float4* out_rgba, float* out_depth, unsigned char* order, Counters* counters,
                           unsigned int* work) {
    extern __shared__ float4 s_tf[];
    for (int i = threadIdx.x; i < P.ntf; i += blockDim.x) s_tf[i] = tf[i];
    __syncthreads();
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const unsigned below = (1u << lane) - 1u;
    const int ntiles = P.ntx * P.nty;
    const unsigned wpt = (unsigned)(P.tp >> 5);              // warps per tile
    const unsigned n_units = (unsigned)(P.ncam * ntiles) * wpt;
    unsigned unit = 0;                                       // the warp's share of pixels (warp-uniform)
    int upos = 32;                                           // its next unassigned pixel
    bool drained = false;
    // the lane's ray
    bool live = false, seg = false, stop = false;
    int c = 0, ct = 0, px = 0, py = 0, depth_key = KEY_EMPTY, last = -1, i = 0;
    float C0 = 0.f, C1 = 0.f, C2 = 0.f, Tr = 1.0f, Tb = 1.0f;
    // its open segment: brick, sample range and local frame, next sample
    int bi = 0, k = 0;
    MarchState m;
    unsigned long long nsamp = 0;
    for (;;) {
        // free lanes take the next pixels of the warp's share (a new share
        // from the counter when it is used up)
        unsigned idle = __ballot_sync(FULL, !live);
        if (__popc(idle) >= REFILL_AT || idle == FULL) {
            while (idle != 0u && !drained) {
                if (upos == 32) {
                    unsigned u = 0;
                    if (lane == 0) u = atomicAdd(work, 1u);
                    u = __shfl_sync(FULL, u, 0);
                    if (u >= n_units) {
                        drained = true;
                        break;
                    }
                    unit = u;
                    upos = 0;
                }
                const int r = __popc(idle & below);
                const bool mine = ((idle >> lane) & 1u) && r < 32 - upos;
                if (mine) {
                    ct = (int)(unit / wpt);
                    c = ct / ntiles;
                    const int tile = ct % ntiles;
                    int lx, ly;
                    tile_pixel((int)((unit % wpt) * 32) + upos + r, P.tw, lx, ly);
                    px = (tile % P.ntx) * P.tw + lx;
                    py = (tile / P.ntx) * P.th + ly;
                    if (px < P.W && py < P.H) {
                        live = true;
                        seg = stop = false;
                        depth_key = KEY_EMPTY;
                        last = -1;
                        i = 0;
                        C0 = C1 = C2 = 0.f;
                        Tr = 1.0f;
                    }
                }
                upos = min(32, upos + __popc(idle));
                idle &= ~__ballot_sync(FULL, mine);
            }
        }
        const unsigned marching = __ballot_sync(FULL, live);
        if (marching == 0u) {
            if (drained) break;
            continue;
        }
        unsigned char* ord = nullptr;
        if (live && order) ord = order + (((long long)c * P.H + py) * P.W + px) * P.order_stride;
        if (live && !seg) {
            // the ray's next brick segment front to back
            long long first = tile_first[ct];
            int cnt = tile_count[ct];
            if (first < 0 || first + cnt > P.items_cap) cnt = 0;     // list overflowed: error bit already set
            int j0;
            const int q = next_segment(P, cams[c], c, bricks, items, first, cnt, px, py, last, j0);
            if (q < 0) {
                // the ray is done: its pixel
                if (ord)
                    for (; i < P.order_stride; ++i) ord[i] = 0xFF;
                write_pixel(P, cams[c], c, px, py, C0, C1, C2, Tr, depth_key, out_rgba, out_depth);
                live = false;
            } else {
                last = j0;
                const Item it = items[first + q];
                if (ord && i < P.order_stride) ord[i] = (unsigned char)it.brick;
                ++i;
                if (!stop) {                    // behind the termination: listed, not marched
                    bi = it.brick;
                    if (brick_samples(P, cams[c], c, bricks[bi], px, py, m)) {
                        seg = true;
                        k = 0;
                        Tb = Tr;
                    }
                }
            }
        }
        // the open segments, until REFILL_AT lanes have left the march
        const int keep = __popc(__ballot_sync(FULL, seg)) - REFILL_AT + 1;
        if (seg) {
            const BrickDev& b = bricks[bi];
            const int st = march_resume<T, GL, SKIP>(P, b, scales[b.scale_idx], s_tf, m, keep, k, C0, C1, C2, Tr,
                                                     nsamp);
            if (st != 0) {
                seg = false;
                if (Tr < Tb && depth_key == KEY_EMPTY) depth_key = m.j0;
                if (st == 2) {
                    stop = true;
                    if (!ord) {                 // terminated, no order map to finish
                        write_pixel(P, cams[c], c, px, py, C0, C1, C2, Tr, depth_key, out_rgba, out_depth);
                        live = false;
                    }
                }
            }
        }
    }
    nsamp = warp_sum_u64(nsamp);
    if (lane == 0 && nsamp) atomicAdd(&counters->samples_fwd, nsamp);
}

template <typename T, int GL, bool SKIP>
static void ordered_launch_s(const FrameParams& P, const CamBasis* cams, const BrickDev* bricks, const float* scales,
                             const int* tile_first, const int* tile_count, const Item* items, const float4* tf,
                             float4* out_rgba, float* out_depth, unsigned char* order, Counters* counters,
                             unsigned int* work, cudaStream_t st) {
    size_t smem = sizeof(float4) * P.ntf;
    if (work) {
        auto kern = k_march_ordered_refill<T, GL, SKIP>;
        if (smem > 48 * 1024) cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        int per_sm = 0, dev = 0, nsm = 148;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, P.tp, smem);
        const int nct = P.ncam * P.ntx * P.nty;
        const int grid = std::min(nsm * std::max(per_sm, 1), nct);
        cudaMemsetAsync(work, 0, sizeof(unsigned int), st);
        kern<<<grid, P.tp, smem, st>>>(P, cams, bricks, scales, tile_first, tile_count, items, tf, out_rgba,
                                       out_depth, order, counters, work);
        return;
    }
    if (smem > 48 * 1024)
        cudaFuncSetAttribute(k_march_ordered<T, GL, SKIP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    const int nct = P.ncam * P.ntx * P.nty;
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
