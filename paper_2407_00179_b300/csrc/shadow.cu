// shadow.cu -- volumetric shadows by ray forwarding between bricks.
//
// Every primary sample of every brick's ray segment spawns one shadow ray
// toward the directional light.  The shadow rays form one wave-front per
// brick (the rays its own samples spawned, records contiguous in the
// brick-major work order).  In K rounds, round r lets brick (w + r) mod K
// march every ray of wave-front w through the samples it owns, multiplying
// the ray's transmittance: the ring exchange of full wave-fronts the paper
// adopts for data-parallel ray tracing (§2.3), with each brick reading only
// its own stored nodes.  After the K rounds every ray has met every brick;
// the shading march then scales each sample's emission by
// k_a + (1 - k_a) T_light and writes ordinary per-brick fragments for the
// sort-last compositor.
//
// Shadow sample i of a ray from p lies at p + (i + 1/2) h L (node units).
// A brick evaluates the samples whose FP32 position lies in its owned
// region (the partition rule of the primary march: half-open, closed at the
// volume's upper faces), so every position inside the volume box has
// exactly one owner and a position outside none: the ray ends where it
// leaves the box.
#include <algorithm>

#include "dpv_internal.cuh"
#include "launch.h"

namespace dpv {

namespace {

// Samples of the primary ray of (item, thread) in its brick: the record
// count of the slot.  Slots follow the brick-major order `sched`.
__global__ void __launch_bounds__(256) k_shadow_count(FrameParams P, const CamBasis* cams, const BrickDev* bricks,
                                                      const Item* items, const int* sched, int* counts) {
    const int i = blockIdx.x;
    const Item it = items[sched[i]];
    int n = 0;
    if (item_ok(it, P)) {
        int lx, ly;
        tile_pixel(threadIdx.x, P.tw, lx, ly);
        const int px = (it.tile % P.ntx) * P.tw + lx, py = (it.tile / P.ntx) * P.th + ly;
        MarchState m;
        if (px < P.W && py < P.H && brick_samples(P, cams[it.cam], it.cam, bricks[it.brick], px, py, m))
            n = m.j1 - m.j0;
    }
    counts[(long long)i * P.tp + threadIdx.x] = n;
}

// Exclusive scan of int counts into 64-bit offsets, in chunks of 1024: each
// block scans its chunk and writes the chunk's sum; one block scans the
// sums; a last pass adds each chunk's base.
__device__ __forceinline__ long long block_exclusive_scan(long long v, long long* s_warp, long long& total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    long long x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const long long y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_warp[warp] = x;
    __syncthreads();
    if (warp == 0) {
        long long w = lane < (int)(blockDim.x >> 5) ? s_warp[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const long long y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        s_warp[lane] = w;                    // inclusive sums of the warps
    }
    __syncthreads();
    total = s_warp[(blockDim.x >> 5) - 1];
    const long long before = warp > 0 ? s_warp[warp - 1] : 0;
    __syncthreads();
    return before + x - v;
}

__global__ void __launch_bounds__(1024) k_scan_chunks(const int* in, long long n, long long* out, long long* sums) {
    __shared__ long long s_warp[32];
    const long long i = (long long)blockIdx.x * 1024 + threadIdx.x;
    const long long v = i < n ? in[i] : 0;
    long long total;
    const long long e = block_exclusive_scan(v, s_warp, total);
    if (i < n) out[i] = e;
    if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

__global__ void __launch_bounds__(1024) k_scan_sums(long long* sums, int n, long long* total_out) {
    __shared__ long long s_warp[32];
    __shared__ long long carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int base = 0; base < n; base += 1024) {
        const int i = base + threadIdx.x;
        const long long v = i < n ? sums[i] : 0;
        long long total;
        const long long e = block_exclusive_scan(v, s_warp, total);
        if (i < n) sums[i] = carry + e;
        __syncthreads();
        if (threadIdx.x == 0) carry += total;
        __syncthreads();
    }
    if (threadIdx.x == 0) *total_out = carry;
}

__global__ void k_scan_add(long long* out, long long n, const long long* sums) {
    const long long i = (long long)blockIdx.x * 1024 + threadIdx.x;
    if (i < n) out[i] += sums[blockIdx.x];
}

// First record of every brick's wave-front: the offset of the brick's first
// slot in the brick-major order (item_first = the schedule's per-brick item
// offsets), and the total at the end.
__global__ void k_wave_first(int nbricks, int tp, const int* item_first, const long long* offsets,
                             const long long* total, int n_items, long long* rec_first) {
    const int b = threadIdx.x + blockIdx.x * blockDim.x;
    if (b > nbricks) return;
    const int i = b < nbricks ? item_first[b] : n_items;
    rec_first[b] = i < n_items ? offsets[(long long)i * tp] : *total;
}

// One record per primary sample: its global node position and T = 1.
__global__ void __launch_bounds__(256) k_shadow_spawn(FrameParams P, const CamBasis* cams, const BrickDev* bricks,
                                                      const Item* items, const int* sched,
                                                      const long long* offsets, float4* recs) {
    const int i = blockIdx.x;
    const Item it = items[sched[i]];
    if (!item_ok(it, P)) return;
    int lx, ly;
    tile_pixel(threadIdx.x, P.tw, lx, ly);
    const int px = (it.tile % P.ntx) * P.tw + lx, py = (it.tile / P.ntx) * P.th + ly;
    if (px >= P.W || py >= P.H) return;
    const BrickDev b = bricks[it.brick];
    MarchState m;
    if (!brick_samples(P, cams[it.cam], it.cam, b, px, py, m)) return;
    float4* out = recs + offsets[(long long)i * P.tp + threadIdx.x];
    const float o0 = (float)b.s_lo[0], o1 = (float)b.s_lo[1], o2 = (float)b.s_lo[2];
    for (int k = 0; k < m.j1 - m.j0; ++k) {
        const float fk = (float)k;
        out[k] = make_float4(o0 + fmaf(fk, m.st[0], m.q0[0]), o1 + fmaf(fk, m.st[1], m.q0[1]),
                             o2 + fmaf(fk, m.st[2], m.q0[2]), 1.0f);
    }
}

// Does brick b own global node-space position p?
__device__ __forceinline__ bool owns(const BrickDev& b, const float p[3]) {
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (p[a] < b.r0[a]) return false;
        if (b.closed[a] ? p[a] > b.r1[a] : p[a] >= b.r1[a]) return false;
    }
    return true;
}

// Round r: brick (w + r) mod K marches every ray of wave-front w through
// the shadow samples it owns.  One grid covers the records of all
// wave-fronts evenly (wave-fronts differ in size); a record's wave-front is
// found in the K + 1 first-record offsets.
// the pipelined cell-layout round at 4 CTAs per SM (64 registers): 7 %
// faster than the plain loop at 5
template <int GL>
constexpr int shadow_min_ctas() {
    return GL == GATHER_CELL ? 4 : 1;
}

template <typename T, int GL>
__global__ void __launch_bounds__(256, shadow_min_ctas<GL>()) k_shadow_round(FrameParams P, const BrickDev* bricks, const float* scales,
                                                      const float4* tf, const long long* rec_first, int round,
                                                      float4* recs, Counters* counters) {
    extern __shared__ float4 s_tf[];
    __shared__ long long s_first[MAX_RANKS + 1];
    for (int i = threadIdx.x; i < P.ntf; i += blockDim.x) s_tf[i] = tf[i];
    for (int i = threadIdx.x; i <= P.nbricks; i += blockDim.x) s_first[i] = rec_first[i];
    __syncthreads();
    const long long total = s_first[P.nbricks];
    const float hl[3] = {P.hl[0], P.hl[1], P.hl[2]};
    unsigned long long nsamp = 0;
    int w = 0;
    for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < total;
         r += (long long)gridDim.x * blockDim.x) {
        while (w + 1 < P.nbricks && r >= s_first[w + 1]) ++w;     // records ascend: w only grows
        const BrickDev& b = bricks[(w + round) % P.nbricks];
        const float scale = scales[b.scale_idx];
        const T* data = (const T*)b.data;
        const int lim[3] = {b.s_n[0] - 2, b.s_n[1] - 2, b.s_n[2] - 2};
        float4 rec = recs[r];
        const float o[3] = {rec.x, rec.y, rec.z};
        // the step interval t (sample i at t = i + 1/2) inside the owned box,
        // widened by one sample each way; ownership is then decided per sample
        float t0 = 0.0f, t1 = 3.0e38f;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            if (hl[a] != 0.0f) {
                const float u0 = (b.r0[a] - o[a]) / hl[a], u1 = (b.r1[a] - o[a]) / hl[a];
                t0 = fmaxf(t0, fminf(u0, u1));
                t1 = fminf(t1, fmaxf(u0, u1));
            } else if (o[a] < b.r0[a] || o[a] > b.r1[a]) {
                t1 = -1.0f;
            }
        }
        if (!(t0 <= t1)) continue;
        const int i0 = max(0, (int)floorf(t0 - 0.5f) - 1);
        const int i1 = (int)fminf(ceilf(t1 - 0.5f) + 1.0f, 1.0e9f);
        float Tl = rec.w;
        CornerCache<T, GL> cc;
        bool any = false;
        if (GL == GATHER_CELL) {
            // the owned samples are one contiguous run (each coordinate of
            // fma(i + 1/2, hL, o) is monotone in i): find its start, then
            // fetch each next sample's cell while this one's is evaluated
            int i = i0;
            float p[3];
            bool own = false;
            for (; i <= i1; ++i) {
                const float ti = (float)i + 0.5f;
                p[0] = fmaf(ti, hl[0], o[0]);
                p[1] = fmaf(ti, hl[1], o[1]);
                p[2] = fmaf(ti, hl[2], o[2]);
                if (owns(b, p)) {
                    own = true;
                    break;
                }
            }
            if (own) {
                CellRaw<T> raw;
                int ix, iy, iz;
                float fx, fy, fz;
                {
                    const float qx = p[0] - (float)b.s_lo[0], qy = p[1] - (float)b.s_lo[1], qz = p[2] - (float)b.s_lo[2];
                    ix = min(max(__float2int_rd(qx), 0), lim[0]);
                    iy = min(max(__float2int_rd(qy), 0), lim[1]);
                    iz = min(max(__float2int_rd(qz), 0), lim[2]);
                    fx = qx - (float)ix;
                    fy = qy - (float)iy;
                    fz = qz - (float)iz;
                }
                raw.fetch(b.gather, cell_slot(b, ix, iy, iz));
                for (;;) {
                    float v[8];
                    raw.decode(v);
                    const float cx = fx, cy = fy, cz = fz;
                    bool nown = false;
                    if (i + 1 <= i1) {
                        const float tn = (float)(i + 1) + 0.5f;
                        p[0] = fmaf(tn, hl[0], o[0]);
                        p[1] = fmaf(tn, hl[1], o[1]);
                        p[2] = fmaf(tn, hl[2], o[2]);
                        nown = owns(b, p);
                        if (nown) {
                            const float qx = p[0] - (float)b.s_lo[0], qy = p[1] - (float)b.s_lo[1],
                                        qz = p[2] - (float)b.s_lo[2];
                            ix = min(max(__float2int_rd(qx), 0), lim[0]);
                            iy = min(max(__float2int_rd(qy), 0), lim[1]);
                            iz = min(max(__float2int_rd(qz), 0), lim[2]);
                            fx = qx - (float)ix;
                            fy = qy - (float)iy;
                            fz = qz - (float)iz;
                            raw.fetch(b.gather, cell_slot(b, ix, iy, iz));
                        }
                    }
                    const float s = lerp_cell<T>(v, cx, cy, cz, scale);
                    const TFSample c = tf_lookup(s_tf, P, s);
                    const float al = opacity(P.sigma_max * c.v.w * P.shadow_dt);
                    Tl = Tl * (1.0f - al);
                    ++nsamp;
                    if (!nown) break;
                    ++i;
                }
                recs[r].w = Tl;
            }
            continue;
        }
        for (int i = i0; i <= i1; ++i) {
            const float ti = (float)i + 0.5f;
            const float p[3] = {fmaf(ti, hl[0], o[0]), fmaf(ti, hl[1], o[1]), fmaf(ti, hl[2], o[2])};
            if (!owns(b, p)) continue;
            int ix, iy, iz;
            float fx, fy, fz;
            {
                const float qx = p[0] - (float)b.s_lo[0], qy = p[1] - (float)b.s_lo[1], qz = p[2] - (float)b.s_lo[2];
                ix = min(max(__float2int_rd(qx), 0), lim[0]);
                iy = min(max(__float2int_rd(qy), 0), lim[1]);
                iz = min(max(__float2int_rd(qz), 0), lim[2]);
                fx = qx - (float)ix;
                fy = qy - (float)iy;
                fz = qz - (float)iz;
            }
            const float s = trilinear<T, GL>(b, data, scale, cc, ix, iy, iz, fx, fy, fz);
            const TFSample c = tf_lookup(s_tf, P, s);
            const float al = opacity(P.sigma_max * c.v.w * P.shadow_dt);
            Tl = Tl * (1.0f - al);
            any = true;
            ++nsamp;
        }
        if (any) recs[r].w = Tl;
    }
    nsamp = warp_sum_u64(nsamp);
    if ((threadIdx.x & 31) == 0 && nsamp) atomicAdd(&counters->samples_shadow, nsamp);
}

// The shading march: the sort-last march with each sample's emission scaled
// by k_a + (1 - k_a) T_light (its record); fragments go to the item's slots.
template <typename T, int GL>
__global__ void __launch_bounds__(256) k_march_shadowed(FrameParams P, const CamBasis* cams, const BrickDev* bricks,
                                                        const float* scales, const Item* items, const int* sched,
                                                        const long long* offsets, const float4* recs,
                                                        const float4* tf, float4* frag_rgba, int* frag_key,
                                                        Counters* counters) {
    extern __shared__ float4 s_tf[];
    for (int i = threadIdx.x; i < P.ntf; i += blockDim.x) s_tf[i] = tf[i];
    __syncthreads();
    const int i = blockIdx.x;
    const int item = sched[i];
    const Item it = items[item];
    if (!item_ok(it, P)) return;
    const BrickDev b = bricks[it.brick];
    const CamBasis cam = cams[it.cam];
    const float scale = scales[b.scale_idx];
    const T* data = (const T*)b.data;
    int lx, ly;
    tile_pixel(threadIdx.x, P.tw, lx, ly);
    const int px = (it.tile % P.ntx) * P.tw + lx, py = (it.tile / P.ntx) * P.th + ly;
    const long long slot = (long long)item * P.tp + threadIdx.x;
    unsigned long long nsamp = 0;
    if (px < P.W && py < P.H) {
        MarchState m;
        if (brick_samples(P, cam, it.cam, b, px, py, m)) {
            const float4* rec = recs + offsets[(long long)i * P.tp + threadIdx.x];
            float C0 = 0.f, C1 = 0.f, C2 = 0.f, Tr = 1.0f;
            const int n = m.j1 - m.j0;
            CornerCache<T, GL> cc;
            SampleWalker wk;
            wk.init(b);
            for (int k = 0; k < n; ++k) {
                int ix, iy, iz;
                float fx, fy, fz;
                wk.at(m, k, ix, iy, iz, fx, fy, fz);
                ++nsamp;
                const float s = trilinear<T, GL>(b, data, scale, cc, ix, iy, iz, fx, fy, fz);
                const TFSample c = tf_lookup(s_tf, P, s);
                const float al = sample_alpha(P, c.v.w);
                const float light = fmaf(1.0f - P.ambient, rec[k].w, P.ambient);
                const float ta = Tr * al * light;
                C0 = fmaf(ta, c.v.x, C0);
                C1 = fmaf(ta, c.v.y, C1);
                C2 = fmaf(ta, c.v.z, C2);
                Tr = Tr - Tr * al;     // the unshadowed frame's update, bit for bit
                if (P.ert_on && 1.0f - Tr > P.ert) break;
            }
            frag_rgba[slot] = make_float4(C0, C1, C2, 1.0f - Tr);
            frag_key[slot] = m.j0;
        } else {
            frag_key[slot] = KEY_EMPTY;
        }
    }
    nsamp = warp_sum_u64(nsamp);
    if ((threadIdx.x & 31) == 0 && nsamp) atomicAdd(&counters->samples_fwd, nsamp);
}

template <typename T, int GL>
void rounds_and_shade(const FrameParams& P, const CamBasis* cams, const BrickDev* bricks, const float* scales,
                      const Item* items, int n_items, const int* sched, const long long* offsets,
                      const long long* rec_first, long long n_recs, float4* recs, const float4* tf,
                      float4* frag_rgba, int* frag_key, Counters* counters, cudaStream_t st) {
    const size_t smem = sizeof(float4) * P.ntf;
    if (smem > 48 * 1024) {
        cudaFuncSetAttribute(k_shadow_round<T, GL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        cudaFuncSetAttribute(k_march_shadowed<T, GL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    }
    // one grid over every wave-front's records: 16 CTAs of 256 per SM
    const int grid = (int)std::max<long long>(1, std::min<long long>((n_recs + 255) / 256, 148LL * 16));
    for (int r = 0; r < P.nbricks; ++r)
        k_shadow_round<T, GL><<<grid, 256, smem, st>>>(P, bricks, scales, tf, rec_first, r, recs, counters);
    k_march_shadowed<T, GL><<<n_items, P.tp, smem, st>>>(P, cams, bricks, scales, items, sched, offsets, recs, tf,
                                                         frag_rgba, frag_key, counters);
}

}  // namespace

cudaError_t launch_shadow_offsets(const FrameParams& P, const CamBasis* cams, const BrickDev* bricks,
                                  const Item* items, int n_items, const int* sched, int* counts, long long* offsets,
                                  long long* chunk_sums, long long* total, cudaStream_t st) {
    if (n_items <= 0) return cudaMemsetAsync(total, 0, sizeof(long long), st);
    const long long n = (long long)n_items * P.tp;
    const int chunks = (int)((n + 1023) / 1024);
    k_shadow_count<<<n_items, P.tp, 0, st>>>(P, cams, bricks, items, sched, counts);
    k_scan_chunks<<<chunks, 1024, 0, st>>>(counts, n, offsets, chunk_sums);
    k_scan_sums<<<1, 1024, 0, st>>>(chunk_sums, chunks, total);
    k_scan_add<<<chunks, 1024, 0, st>>>(offsets, n, chunk_sums);
    return cudaGetLastError();
}

size_t shadow_chunk_count(const FrameParams& P, int n_items) {
    return (size_t)(((long long)std::max(1, n_items) * P.tp + 1023) / 1024);
}

cudaError_t launch_shadow_render(int dtype, int gather, const FrameParams& P, const CamBasis* cams,
                                 const BrickDev* bricks, const float* scales, const Item* items, int n_items,
                                 const int* sched, const int* item_first, const long long* offsets,
                                 const long long* total, long long* rec_first, long long n_recs, float4* recs,
                                 const float4* tf, float4* frag_rgba, int* frag_key, Counters* counters,
                                 cudaStream_t st) {
    if (n_items <= 0) return cudaSuccess;
    k_wave_first<<<(P.nbricks + 1 + 255) / 256, 256, 0, st>>>(P.nbricks, P.tp, item_first, offsets, total, n_items,
                                                             rec_first);
    k_shadow_spawn<<<n_items, P.tp, 0, st>>>(P, cams, bricks, items, sched, offsets, recs);
#define SHADE(T, GL)                                                                                          \
    rounds_and_shade<T, GL>(P, cams, bricks, scales, items, n_items, sched, offsets, rec_first, n_recs, recs, \
                            tf, frag_rgba, frag_key, counters, st)
#define SHADE_T(T)                                                                                            \
    (gather == GATHER_CELL ? SHADE(T, GATHER_CELL) : gather == GATHER_QUAD ? SHADE(T, GATHER_QUAD)           \
                                                                           : SHADE(T, GATHER_LINEAR))
    switch (dtype) {
        case 0: SHADE_T(float); break;
        case 1: SHADE_T(__half); break;
        case 2: SHADE_T(__nv_bfloat16); break;
        default: SHADE_T(__nv_fp8_e4m3); break;
    }
#undef SHADE_T
#undef SHADE
    return cudaGetLastError();
}

}  // namespace dpv
