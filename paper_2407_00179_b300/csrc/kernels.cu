// kernels.cu -- the GPU path: brick commit, culling / work list, brick
// ray-march, sort-last compositor, and their adjoints (sm_103a).
//
// Paper structure followed (arXiv 2407.00179): every rank owns one spatial
// part of the volume (§1, §3.1.2) with a ghost layer (§1); each rank reduces
// its part to one RGBA fragment per pixel, which is exact for convex parts
// (§2.1); fragments carry a depth key and are sorted per pixel and blended
// front to back in one kernel (§5.1.1, "Compositing").  The paper's parallel
// direct send is replaced by the compositor reading every logical rank's
// fragments straight from HBM.
#include <stdlib.h>

#include <algorithm>
#include <type_traits>

#include "dpv_internal.cuh"
#include "launch.h"

namespace dpv {

// ===========================================================================
// brick commit (ghost extraction + storage conversion)
// ===========================================================================

template <typename T>
__device__ __forceinline__ float src_value(const T* p, long long i);
template <>
__device__ __forceinline__ float src_value<float>(const float* p, long long i) { return p[i]; }

template <typename T>
__device__ __forceinline__ T to_storage(float v);
template <>
__device__ __forceinline__ float to_storage<float>(float v) { return v; }
template <>
__device__ __forceinline__ __half to_storage<__half>(float v) { return __float2half_rn(v); }
template <>
__device__ __forceinline__ __nv_bfloat16 to_storage<__nv_bfloat16>(float v) { return __float2bfloat16_rn(v); }
template <>
__device__ __forceinline__ __nv_fp8_e4m3 to_storage<__nv_fp8_e4m3>(float v) {
    __nv_fp8_e4m3 r;
    r.__x = __nv_cvt_float_to_fp8(v, __NV_SATFINITE, __NV_E4M3);
    return r;
}

// Linear index in the source box of stored node k of a brick.
__device__ __forceinline__ long long src_index(long long k, const CommitArgs& a) {
    long long nx = a.s_n[0], nxy = (long long)a.s_n[0] * a.s_n[1];
    long long z = k / nxy, y = (k - z * nxy) / nx, x = k - z * nxy - y * nx;
    long long gx = x + a.s_lo[0] - a.d_lo[0], gy = y + a.s_lo[1] - a.d_lo[1], gz = z + a.s_lo[2] - a.d_lo[2];
    return (gz * a.d_n[1] + gy) * (long long)a.d_n[0] + gx;
}

// max |v| over the stored nodes (non-negative floats order like their bits)
__global__ void k_brick_maxabs(CommitArgs a, unsigned int* out) {
    long long n = (long long)a.s_n[0] * a.s_n[1] * a.s_n[2];
    float m = 0.0f;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x)
        m = fmaxf(m, fabsf(src_value<float>((const float*)a.src, src_index(k, a))));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out, __float_as_uint(m));
}

// scale = given, or max|v| / 448 for fp8 (1 if zero), or 1
__global__ void k_brick_scale(const unsigned int* maxabs, float given, int fp8, float* scale_out) {
    float s = given;
    if (!(given > 0.0f)) {
        s = 1.0f;
        if (fp8) {
            float m = __uint_as_float(*maxabs);
            if (m > 0.0f) s = m / 448.0f;
        }
    }
    *scale_out = s;
}

template <typename T>
__global__ void k_brick_convert(CommitArgs a, const float* scale, T* dst) {
    long long n = (long long)a.s_n[0] * a.s_n[1] * a.s_n[2];
    float sc = *scale;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
        float v = src_value<float>((const float*)a.src, src_index(k, a));
        dst[k] = to_storage<T>(v / sc);
    }
}

// same-format copy (no conversion), element size es
__global__ void k_brick_copy(CommitArgs a, int es, unsigned char* dst) {
    long long n = (long long)a.s_n[0] * a.s_n[1] * a.s_n[2];
    const unsigned char* s = (const unsigned char*)a.src;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
        long long si = src_index(k, a);
        for (int b = 0; b < es; ++b) dst[k * es + b] = s[si * es + b];
    }
}

cudaError_t launch_commit(const CommitArgs& a, int storage, int src_is_f32, float given_scale, unsigned int* d_tmp,
                          float* d_scale, void* dst, cudaStream_t st) {
    long long n = (long long)a.s_n[0] * a.s_n[1] * a.s_n[2];
    long long nb = (n + 255) / 256;
    int blocks = (int)(nb < 148LL * 16 ? nb : 148LL * 16);
    if (!src_is_f32) {
        // data already in the storage format: copy, scale as given (default 1)
        k_brick_scale<<<1, 1, 0, st>>>(d_tmp, given_scale, 0, d_scale);
        static const int es[4] = {4, 2, 2, 1};
        k_brick_copy<<<blocks, 256, 0, st>>>(a, es[storage], (unsigned char*)dst);
        return cudaGetLastError();
    }
    cudaMemsetAsync(d_tmp, 0, sizeof(unsigned int), st);
    if (storage == 3 && !(given_scale > 0.0f)) k_brick_maxabs<<<blocks, 256, 0, st>>>(a, d_tmp);
    k_brick_scale<<<1, 1, 0, st>>>(d_tmp, given_scale, storage == 3, d_scale);
    switch (storage) {
        case 0: k_brick_convert<float><<<blocks, 256, 0, st>>>(a, d_scale, (float*)dst); break;
        case 1: k_brick_convert<__half><<<blocks, 256, 0, st>>>(a, d_scale, (__half*)dst); break;
        case 2: k_brick_convert<__nv_bfloat16><<<blocks, 256, 0, st>>>(a, d_scale, (__nv_bfloat16*)dst); break;
        default: k_brick_convert<__nv_fp8_e4m3><<<blocks, 256, 0, st>>>(a, d_scale, (__nv_fp8_e4m3*)dst); break;
    }
    return cudaGetLastError();
}

// ===========================================================================
// cameras and culling (work list)
// ===========================================================================

__global__ void k_cam_setup(const CamIn* cams, int n, float3 origin, float spacing, int H, CamBasis* out,
                            CamBasisDF* outd) {
    // once per camera, so computed in FP64 and rounded once to FP32 (and to
    // double-float for the ray setup)
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    CamIn c = cams[i];
    double f[3] = {(double)c.center[0] - c.eye[0], (double)c.center[1] - c.eye[1], (double)c.center[2] - c.eye[2]};
    double fn = 1.0 / sqrt(f[0] * f[0] + f[1] * f[1] + f[2] * f[2]);
    for (int a = 0; a < 3; ++a) f[a] *= fn;
    double up[3] = {c.up[0], c.up[1], c.up[2]};
    double r[3] = {f[1] * up[2] - f[2] * up[1], f[2] * up[0] - f[0] * up[2], f[0] * up[1] - f[1] * up[0]};
    double rn = 1.0 / sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
    for (int a = 0; a < 3; ++a) r[a] *= rn;
    double u[3] = {r[1] * f[2] - r[2] * f[1], r[2] * f[0] - r[0] * f[2], r[0] * f[1] - r[1] * f[0]};
    CamBasis b;
    const double og[3] = {origin.x, origin.y, origin.z};
    double o[3];
    for (int a = 0; a < 3; ++a) {
        o[a] = ((double)c.eye[a] - og[a]) / (double)spacing;
        b.o[a] = (float)o[a];
        b.f[a] = (float)f[a];
        b.r[a] = (float)r[a];
        b.u[a] = (float)u[a];
    }
    double th = tan((double)c.fovy_deg * 0.00872664625997164788);   // pi / 360
    b.th = (float)th;
    b.pad = 0.0f;
    out[i] = b;
    CamBasisDF bd;
    for (int a = 0; a < 3; ++a) {
        bd.o[a] = df_of(o[a]);
        bd.f[a] = df_of(f[a]);
        bd.r[a] = df_of(r[a]);
        bd.u[a] = df_of(u[a]);
    }
    bd.k = df_of(th / (double)H);
    bd.inv_spacing = df_of(1.0 / (double)spacing);
    outd[i] = bd;
}

// Ray setup: direction of every pixel's ray, normalize(f + x th r + y th u)
// with x = ((px + 1/2) / W * 2 - 1) * W / H and y = (py + 1/2) / H * 2 - 1
// (that is x th = (2 px + 1 - W) th / H, y th = (2 py + 1 - H) th / H),
// scaled to node units per world t, in double-float arithmetic (the norm by
// an FP32 reciprocal square root and one Newton step).  Stored per ray
// (RAY_VECS float4):
//   0: direction rounded to FP32, t_enter      (FP32, from the FP32 slab)
//   1: FP32 reciprocal direction, t_exit
//   2: entry point eye + t_enter d, high FP32 part (double-float slab and
//      product)
//   3: entry point, low part
//   4: direction, low part
// The FP32 parts fix the sample ranges (identical planes in every kernel);
// the pairs place each brick's first sample accurately.
__global__ void k_rays(FrameParams P, const CamBasis* cams, const CamBasisDF* camd, float4* rays) {
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    long long npix = (long long)P.W * P.H;
    if (i >= npix * P.ncam) return;
    int c = (int)(i / npix);
    int p = (int)(i - c * npix);
    int px = p % P.W, py = p / P.W;
    const CamBasisDF& b = camd[c];
    const DF x = df_mulf(b.k, (float)(2 * px + 1 - P.W));
    const DF y = df_mulf(b.k, (float)(2 * py + 1 - P.H));
    DF d[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) d[a] = df_add(b.f[a], df_add(df_mul(x, b.r[a]), df_mul(y, b.u[a])));
    const DF n2 = df_add(df_add(df_mul(d[0], d[0]), df_mul(d[1], d[1])), df_mul(d[2], d[2]));
    const DF n = df_mul(df_rsqrt(n2), b.inv_spacing);
    DF dd[3];
    Ray r;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        dd[a] = df_mul(d[a], n);
        r.d[a] = dd[a].hi;                 // the FP32 rounding of the direction
        r.o[a] = cams[c].o[a];
        r.inv[a] = 1.0f / r.d[a];
    }
    if (!volume_interval(P.dims, r.o, r.d, r.inv, r.te, r.tx)) r.te = r.tx = 0.0f;
    // accurate entry point: slab against [0, dims - 1] with the double-float ray
    DF te = DF{0.0f, 0.0f};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (dd[a].hi != 0.0f) {
            const DF inv = df_rcp(dd[a]);
            const DF ta = df_mul(df_neg(b.o[a]), inv);
            const DF tb = df_mul(df_add(DF{(float)(P.dims[a] - 1), 0.0f}, df_neg(b.o[a])), inv);
            const DF near = df_lt(ta, tb) ? ta : tb;
            if (df_lt(te, near)) te = near;
        }
    }
    float ph[3], pl[3], dl[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const DF pe = df_add(b.o[a], df_mul(te, dd[a]));
        ph[a] = pe.hi;
        pl[a] = pe.lo;
        dl[a] = dd[a].lo;
    }
    float4* o = rays + RAY_VECS * i;
    o[0] = make_float4(r.d[0], r.d[1], r.d[2], r.te);
    o[1] = make_float4(r.inv[0], r.inv[1], r.inv[2], r.tx);
    o[2] = make_float4(ph[0], ph[1], ph[2], 0.0f);
    o[3] = make_float4(pl[0], pl[1], pl[2], 0.0f);
    o[4] = make_float4(dl[0], dl[1], dl[2], 0.0f);
}

// Screen tile rectangle [x0, x1] x [y0, y1] (inclusive) that may see brick b
// from camera c: the bounding box of the projected corners of its owned
// region, one pixel wider on each side.  Corners at or behind the eye plane
// make the rectangle the whole screen; a brick wholly behind is culled.
__global__ void k_cull_rects(FrameParams P, const CamBasis* cams, const BrickDev* bricks, int4* rects) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P.ncam * P.nbricks) return;
    int c = i / P.nbricks, k = i % P.nbricks;
    CamBasis cb = cams[c];
    BrickDev b = bricks[k];
    float aspect = (float)P.W / (float)P.H;
    float xmin = 1e30f, xmax = -1e30f, ymin = 1e30f, ymax = -1e30f;
    int behind = 0, front = 0;
    for (int m = 0; m < 8; ++m) {
        float p[3] = {(m & 1) ? b.r1[0] : b.r0[0], (m & 2) ? b.r1[1] : b.r0[1], (m & 4) ? b.r1[2] : b.r0[2]};
        float v[3] = {p[0] - cb.o[0], p[1] - cb.o[1], p[2] - cb.o[2]};
        float z = v[0] * cb.f[0] + v[1] * cb.f[1] + v[2] * cb.f[2];
        float len = sqrtf(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
        if (z <= 1e-3f * len) {
            ++behind;
            continue;
        }
        ++front;
        float x = (v[0] * cb.r[0] + v[1] * cb.r[1] + v[2] * cb.r[2]) / (z * cb.th * aspect);
        float y = (v[0] * cb.u[0] + v[1] * cb.u[1] + v[2] * cb.u[2]) / (z * cb.th);
        float px = (x + 1.0f) * 0.5f * P.W - 0.5f, py = (y + 1.0f) * 0.5f * P.H - 0.5f;
        xmin = fminf(xmin, px);
        xmax = fmaxf(xmax, px);
        ymin = fminf(ymin, py);
        ymax = fmaxf(ymax, py);
    }
    int4 r;
    if (front == 0) {
        r = make_int4(1, 1, 0, 0);   // empty
    } else if (behind > 0) {
        r = make_int4(0, 0, P.ntx - 1, P.nty - 1);
    } else {
        xmin -= 1.0f;
        ymin -= 1.0f;
        xmax += 1.0f;
        ymax += 1.0f;
        if (xmax < 0.0f || ymax < 0.0f || xmin > (float)(P.W - 1) || ymin > (float)(P.H - 1)) {
            r = make_int4(1, 1, 0, 0);
        } else {
            int x0 = max(0, (int)floorf(fmaxf(xmin, 0.0f)) / P.tw), x1 = min(P.ntx - 1, (int)floorf(fminf(xmax, (float)P.W)) / P.tw);
            int y0 = max(0, (int)floorf(fmaxf(ymin, 0.0f)) / P.th), y1 = min(P.nty - 1, (int)floorf(fminf(ymax, (float)P.H)) / P.th);
            r = make_int4(x0, y0, x1, y1);
        }
    }
    rects[i] = r;
}

__device__ __forceinline__ bool rect_has(int4 r, int tx, int ty) {
    return tx >= r.x && tx <= r.z && ty >= r.y && ty <= r.w;
}

__global__ void k_cull_count(FrameParams P, const int4* rects, int* tile_count) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    int ntiles = P.ntx * P.nty;
    if (i >= P.ncam * ntiles) return;
    int c = i / ntiles, t = i % ntiles, tx = t % P.ntx, ty = t / P.ntx;
    int n = 0;
    for (int k = 0; k < P.nbricks; ++k) n += rect_has(rects[c * P.nbricks + k], tx, ty);
    tile_count[i] = n;
}

// Exclusive scan of n ints by one block; writes the total to *total.
__global__ void k_scan(const int* in, int* out, int n, unsigned long long* total, unsigned int* max_out) {
    __shared__ int warp_sums[32];
    __shared__ int carry;
    __shared__ unsigned int mx;
    if (threadIdx.x == 0) {
        carry = 0;
        mx = 0;
    }
    __syncthreads();
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int base = 0; base < n; base += blockDim.x) {
        int i = base + threadIdx.x;
        int v = i < n ? in[i] : 0;
        if (v > 0) atomicMax(&mx, (unsigned)v);
        int x = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) warp_sums[wid] = x;
        __syncthreads();
        if (wid == 0) {
            int w = lane < nw ? warp_sums[lane] : 0;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                int y = __shfl_up_sync(0xffffffffu, w, o);
                if (lane >= o) w += y;
            }
            if (lane < nw) warp_sums[lane] = w;
        }
        __syncthreads();
        int excl = x - v + (wid > 0 ? warp_sums[wid - 1] : 0) + carry;
        if (i < n) out[i] = excl;
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) carry = excl + v;
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        *total = (unsigned long long)carry;
        if (max_out) *max_out = mx;
    }
}

__global__ void k_cull_fill(FrameParams P, const int4* rects, const int* tile_first, const int* tile_count,
                            Item* items, int cap, unsigned int* err) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    int ntiles = P.ntx * P.nty;
    if (i >= P.ncam * ntiles) return;
    int c = i / ntiles, t = i % ntiles, tx = t % P.ntx, ty = t / P.ntx;
    int f = tile_first[i];
    if (f + tile_count[i] > cap) {
        atomicOr(err, ERR_ITEM_OVERFLOW);
        return;
    }
    for (int k = 0; k < P.nbricks; ++k)
        if (rect_has(rects[c * P.nbricks + k], tx, ty)) {
            Item it;
            it.cam = c;
            it.tile = t;
            it.brick = k;
            it.pad = 0;
            items[f++] = it;
        }
}

cudaError_t launch_cull(const FrameParams& P, const CamIn* d_cam_in, float3 origin, float spacing,
                        CamBasis* d_cams, CamBasisDF* d_camd, float4* d_rays, const BrickDev* d_bricks,
                        int4* d_rects, int* d_tile_count, int* d_tile_first, Item* d_items, int cap,
                        Counters* d_counters, bool fill, cudaStream_t st) {
    k_cam_setup<<<(P.ncam + 63) / 64, 64, 0, st>>>(d_cam_in, P.ncam, origin, spacing, P.H, d_cams, d_camd);
    if (fill) {
        long long n = (long long)P.ncam * P.W * P.H;
        k_rays<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(P, d_cams, d_camd, d_rays);
    }
    int ncb = P.ncam * P.nbricks;
    k_cull_rects<<<(ncb + 127) / 128, 128, 0, st>>>(P, d_cams, d_bricks, d_rects);
    int nct = P.ncam * P.ntx * P.nty;
    k_cull_count<<<(nct + 127) / 128, 128, 0, st>>>(P, d_rects, d_tile_count);
    k_scan<<<1, 1024, 0, st>>>(d_tile_count, d_tile_first, nct, &d_counters->n_items, &d_counters->max_frag);
    if (fill)
        k_cull_fill<<<(nct + 127) / 128, 128, 0, st>>>(P, d_rects, d_tile_first, d_tile_count, d_items, cap,
                                                       &d_counters->err);
    return cudaGetLastError();
}

// ===========================================================================
// brick ray-march (forward)
// ===========================================================================
//
// One CTA per work item (camera, brick, tile); one thread per pixel; warps
// cover 8 x 4 pixel blocks.  Each thread finds its ray's sample range in the
// brick, marches it front to back and writes one fragment (premultiplied
// RGBA, key = first sample index, or key = EMPTY).  The TF table is staged
// in shared memory.

// One work item: every thread marches its pixel's ray through the item's
// brick and writes the fragment to slot `item * tile_pixels + thread`.
// Returns the samples this thread evaluated.
template <typename T, int GL, bool SKIP, bool PAIR = false>
__device__ __forceinline__ unsigned long long march_item(const FrameParams& P, const CamBasis* cams,
                                                         const BrickDev* bricks, const float* scales, const Item& it,
                                                         long long item, int t, const float4* s_tf,
                                                         float4* frag_rgba, int* frag_key) {
    const BrickDev b = bricks[it.brick];
    const CamBasis cam = cams[it.cam];
    const float scale = scales[b.scale_idx];
    const T* data = (const T*)b.data;
    int lx, ly;
    tile_pixel(t, P.tw, lx, ly);
    int px = (it.tile % P.ntx) * P.tw + lx, py = (it.tile / P.ntx) * P.th + ly;
    long long slot = item * P.tp + t;
    unsigned long long nsamp = 0;
    if (px < P.W && py < P.H) {
        MarchState m;
        if (brick_samples(P, cam, it.cam, b, px, py, m)) {
            float C0 = 0.f, C1 = 0.f, C2 = 0.f, Tr = 1.0f;
            int n = m.j1 - m.j0;
            int k = 0;
            CornerCache<T, GL> cc;
            SampleWalker wk;
            wk.init(b);
            int mlast = -1;
            bool mempty = false;
            if ((GL == GATHER_CELL || GL == GATHER_QUAD) && !SKIP && n > 0) {
                // the next sample's cell (or its two faces) is fetched before
                // this one's arithmetic, so its load overlaps the current
                // sample's work; the interpolation is trilinear()'s, bit for bit
                GatherRaw<T, GL == GATHER_CELL ? GATHER_CELL : GATHER_QUAD, PAIR> raw;
                int ix, iy, iz;
                float fx, fy, fz;
                wk.at(m, 0, ix, iy, iz, fx, fy, fz);
                raw.fetch(b, ix, iy, iz);
                // the float32 cell march keeps the TF interval's entries in
                // registers; the others look them up every sample (fewer
                // registers: no spills, 5 CTAs per SM for the quad march)
                typename std::conditional<GL == GATHER_QUAD || sizeof(T) <= 2, TFNoCache, TFCache<false>>::type tfc;
                for (; k < n; ++k) {
                    float v[8];
                    raw.decode(v);
                    const float cx = fx, cy = fy, cz = fz;
                    if (k + 1 < n) {
                        wk.at<!(GL == GATHER_CELL && sizeof(T) == 4)>(m, k + 1, ix, iy, iz, fx, fy, fz);
                        raw.fetch(b, ix, iy, iz);
                    }
                    float s = lerp_cell<T>(v, cx, cy, cz, scale);
                    const float4 c = tfc.lookup(s_tf, P, s);
                    float al = sample_alpha(P, c.w);
                    float ta = Tr * al;
                    C0 = fmaf(ta, c.x, C0);
                    C1 = fmaf(ta, c.y, C1);
                    C2 = fmaf(ta, c.z, C2);
                    Tr = Tr - ta;
                    if (P.ert_on && 1.0f - Tr > P.ert) {
                        ++k;
                        break;
                    }
                }
                nsamp += (unsigned)k;        // the samples evaluated
                n = 0;
            }
            for (; k < n; ++k) {
                int ix, iy, iz;
                float fx, fy, fz;
                wk.at(m, k, ix, iy, iz, fx, fy, fz);
                if (SKIP) {
                    // a transparent macro-cell: opacity 0 leaves C and T exactly as they are
                    const int mi = (iz >> MACRO_SHIFT) * b.mxy + (iy >> MACRO_SHIFT) * b.mx + (ix >> MACRO_SHIFT);
                    if (mi != mlast) {
                        mlast = mi;
                        mempty = b.empty[mi] != 0;
                    }
                    if (mempty) {
                        k = macro_last(m, wk, k, n, ix, iy, iz);   // past the samples left inside
                        continue;
                    }
                }
                ++nsamp;
                float s = trilinear<T, GL>(b, data, scale, cc, ix, iy, iz, fx, fy, fz);
                TFSample c = tf_lookup(s_tf, P, s);
                float al = sample_alpha(P, c.v.w);
                float ta = Tr * al;
                C0 = fmaf(ta, c.v.x, C0);
                C1 = fmaf(ta, c.v.y, C1);
                C2 = fmaf(ta, c.v.z, C2);
                Tr = Tr - ta;
                if (P.ert_on && 1.0f - Tr > P.ert) break;
            }
            frag_rgba[slot] = make_float4(C0, C1, C2, 1.0f - Tr);
            frag_key[slot] = m.j0;
        } else {
            frag_key[slot] = KEY_EMPTY;
        }
    }
    return nsamp;
}

// Deep fragments (DPV_FRAME_DEEP): empty-space skipping splits the brick's
// segment, each run of evaluated samples between transparent macro-cells
// becoming its own fragment with the run's first sample as key (the general
// case of several fragments per pixel from one rank, §2.1, §5.1.1).  Layer
// d of item i is at slot ((i DEEP_LAYERS + d) tp + thread); from the
// DEEP_LAYERS-th run on, the runs continue the last fragment.  Early
// termination stays on the brick's transmittance Tb, as in the sort-last
// march.
template <typename T, int GL>
__device__ __forceinline__ unsigned long long march_item_deep(const FrameParams& P, const CamBasis* cams,
                                                              const BrickDev* bricks, const float* scales,
                                                              const Item& it, long long item, int t,
                                                              const float4* s_tf, float4* frag_rgba, int* frag_key) {
    const BrickDev b = bricks[it.brick];
    const CamBasis cam = cams[it.cam];
    const float scale = scales[b.scale_idx];
    const T* data = (const T*)b.data;
    int lx, ly;
    tile_pixel(t, P.tw, lx, ly);
    int px = (it.tile % P.ntx) * P.tw + lx, py = (it.tile / P.ntx) * P.th + ly;
    const long long base = item * DEEP_LAYERS * P.tp + t;     // layer d at base + d tp
    unsigned long long nsamp = 0;
    if (px < P.W && py < P.H) {
        int nf = 0;
        MarchState m;
        if (brick_samples(P, cam, it.cam, b, px, py, m)) {
            float C0 = 0.f, C1 = 0.f, C2 = 0.f, Tr = 1.0f, Tb = 1.0f;
            const int n = m.j1 - m.j0;
            CornerCache<T, GL> cc;
            SampleWalker wk;
            wk.init(b);
            int mlast = -1;
            bool mempty = false, run = false;
            for (int k = 0; k < n; ++k) {
                int ix, iy, iz;
                float fx, fy, fz;
                wk.at(m, k, ix, iy, iz, fx, fy, fz);
                const int mi = (iz >> MACRO_SHIFT) * b.mxy + (iy >> MACRO_SHIFT) * b.mx + (ix >> MACRO_SHIFT);
                if (mi != mlast) {
                    mlast = mi;
                    mempty = b.empty[mi] != 0;
                }
                if (mempty) {
                    run = false;
                    k = macro_last(m, wk, k, n, ix, iy, iz);
                    continue;
                }
                if (!run && nf < DEEP_LAYERS) {          // a new run: close the last fragment, open one
                    if (nf > 0) frag_rgba[base + (long long)(nf - 1) * P.tp] = make_float4(C0, C1, C2, 1.0f - Tr);
                    frag_key[base + (long long)nf * P.tp] = m.j0 + k;
                    ++nf;
                    C0 = C1 = C2 = 0.0f;
                    Tr = 1.0f;
                }
                run = true;
                ++nsamp;
                float s = trilinear<T, GL>(b, data, scale, cc, ix, iy, iz, fx, fy, fz);
                TFSample c = tf_lookup(s_tf, P, s);
                float al = sample_alpha(P, c.v.w);
                float ta = Tr * al;
                C0 = fmaf(ta, c.v.x, C0);
                C1 = fmaf(ta, c.v.y, C1);
                C2 = fmaf(ta, c.v.z, C2);
                Tr = Tr - ta;
                Tb = Tb - Tb * al;
                if (P.ert_on && 1.0f - Tb > P.ert) break;
            }
            if (nf > 0) frag_rgba[base + (long long)(nf - 1) * P.tp] = make_float4(C0, C1, C2, 1.0f - Tr);
        }
        for (int d = nf; d < DEEP_LAYERS; ++d) frag_key[base + (long long)d * P.tp] = KEY_EMPTY;
    }
    return nsamp;
}

// MODE: 0 the plain march, 1 with empty-space skipping, 2 deep fragments,
// 3 the plain march with the quad layout's pair-wide loads
template <typename T, int GL, int MODE>
__device__ __forceinline__ unsigned long long march_any(const FrameParams& P, const CamBasis* cams,
                                                        const BrickDev* bricks, const float* scales, const Item& it,
                                                        long long item, int t, const float4* s_tf, float4* frag_rgba,
                                                        int* frag_key) {
    if (MODE == 2) return march_item_deep<T, GL>(P, cams, bricks, scales, it, item, t, s_tf, frag_rgba, frag_key);
    return march_item<T, GL, MODE == 1, MODE == 3>(P, cams, bricks, scales, it, item, t, s_tf, frag_rgba, frag_key);
}

// The march over the cell layout is held to 48 registers, 5 CTAs per SM;
// its plain form keeps the next sample's cell in flight (software
// pipelining): more loads in flight per SM, measured 5 % faster than 4 CTAs
// at 52 registers.  The pipelined quad march (plain and pair-wide forms)
// looks its TF entries up from shared memory every sample and fits 48
// registers with no spill, 5 CTAs per SM; keeping the last interval's
// entries in registers instead needs 60 and holds it to 4 (measured: 2048^3
// bf16 193.8 against 194.1 ms, fp8 175.2 against 177.2, 512^3 bf16 2.938
// against 3.007; the lookup without the kept entries at 4 CTAs: 202.5,
// 181.3, 2.954).  The cell march of 16- and 8-bit storage also looks them
// up every sample (its spills at 48 registers go: 2048^3 fp8 181.3 -> 175.7
// ms, 512^3 f16 +1 %); the float32 one keeps them (1.894 against 1.99 ms at
// 512^3).  The others at 64 registers, 4 CTAs per SM.
template <int GL, int MODE>
constexpr int fwd_min_ctas() {
    return GL == GATHER_CELL || (GL == GATHER_QUAD && (MODE == 0 || MODE == 3)) ? 5 : 4;
}

template <typename T, int GL, int MODE>
__global__ void __launch_bounds__(256, fwd_min_ctas<GL, MODE>()) k_march_fwd(FrameParams P, const CamBasis* cams, const BrickDev* bricks,
                                                   const float* scales, const Item* items, const float4* tf,
                                                   float4* frag_rgba, int* frag_key, Counters* counters) {
    extern __shared__ float4 s_tf[];
    for (int i = threadIdx.x; i < P.ntf; i += blockDim.x) s_tf[i] = tf[i];
    __syncthreads();
    const Item it = items[blockIdx.x];
    if (!item_ok(it, P)) return;
    unsigned long long nsamp =
        march_any<T, GL, MODE>(P, cams, bricks, scales, it, blockIdx.x, threadIdx.x, s_tf, frag_rgba, frag_key);
    nsamp = warp_sum_u64(nsamp);
    if ((threadIdx.x & 31) == 0 && nsamp) atomicAdd(&counters->samples_fwd, nsamp);
}

// Persistent form: a grid sized to the GPU whose warps each pull one warp's
// share of a work item (32 pixels of its tile) at a time from a counter, in
// the order `sched` gives (brick-major: all cameras' tiles of one brick
// together, so a brick is read from HBM about once per batch).  A warp
// whose rays are short takes the next unit at once instead of waiting for
// the other warps of its tile, and no barrier separates the units.
template <typename T, int GL, int MODE>
__global__ void __launch_bounds__(256, fwd_min_ctas<GL, MODE>()) k_march_fwd_persistent(FrameParams P, const CamBasis* cams,
                                                              const BrickDev* bricks, const float* scales,
                                                              const Item* items, const int* sched, int n_items,
                                                              unsigned int* work, const float4* tf,
                                                              float4* frag_rgba, int* frag_key, Counters* counters) {
    extern __shared__ float4 s_tf[];
    for (int i = threadIdx.x; i < P.ntf; i += blockDim.x) s_tf[i] = tf[i];
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const unsigned wpt = (unsigned)(P.tp >> 5);               // warps per tile
    const unsigned n_units = (unsigned)n_items * wpt;
    unsigned long long nsamp = 0;
    for (;;) {
        __syncwarp();
        unsigned u = 0;
        if (lane == 0) u = atomicAdd(work, 1u);
        u = __shfl_sync(0xffffffffu, u, 0);
        if (u >= n_units) break;
        const int item = sched[u / wpt];
        const Item it = items[item];
        if (item_ok(it, P))
            nsamp += march_any<T, GL, MODE>(P, cams, bricks, scales, it, item, (int)((u % wpt) * 32 + lane), s_tf,
                                            frag_rgba, frag_key);
    }
    nsamp = warp_sum_u64(nsamp);
    if (lane == 0 && nsamp) atomicAdd(&counters->samples_fwd, nsamp);
}

template <typename T, int GL, int MODE>
static void fwd_launch_s(const FrameParams& P, const CamBasis* cams, const BrickDev* bricks, const float* scales,
                       const Item* items, int n_items, const float4* tf, float4* frag_rgba, int* frag_key,
                       Counters* counters, const Schedule* sch, cudaStream_t st) {
    size_t smem = sizeof(float4) * P.ntf;
    if (sch) {
        if (smem > 48 * 1024)
            cudaFuncSetAttribute(k_march_fwd_persistent<T, GL, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem);
        int per_sm = 0, dev = 0, nsm = 148;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_march_fwd_persistent<T, GL, MODE>, P.tp, smem);
        int grid = nsm * (per_sm > 0 ? per_sm : 1);
        if (sch->ctas_per_sm > 0 && sch->ctas_per_sm < per_sm) grid = nsm * sch->ctas_per_sm;
        if (grid > n_items) grid = n_items;      // a CTA's warps take at least one tile's worth
        cudaMemsetAsync(sch->work, 0, sizeof(unsigned int), st);
        k_march_fwd_persistent<T, GL, MODE><<<grid, P.tp, smem, st>>>(P, cams, bricks, scales, items, sch->sched, n_items,
                                                                  sch->work, tf, frag_rgba, frag_key, counters);
        return;
    }
    if (smem > 48 * 1024)
        cudaFuncSetAttribute(k_march_fwd<T, GL, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_march_fwd<T, GL, MODE><<<n_items, P.tp, smem, st>>>(P, cams, bricks, scales, items, tf, frag_rgba, frag_key,
                                                            counters);
}

// empty-space skipping and deep fragments are template switches: the plain
// march carries no macro-cell test
template <typename T, int GL>
static void fwd_launch(const FrameParams& P, const CamBasis* cams, const BrickDev* bricks, const float* scales,
                       const Item* items, int n_items, const float4* tf, float4* frag_rgba, int* frag_key,
                       Counters* counters, const Schedule* sch, cudaStream_t st) {
    if (P.deep > 1) {
        fwd_launch_s<T, GL, 2>(P, cams, bricks, scales, items, n_items, tf, frag_rgba, frag_key, counters, sch, st);
    } else if (P.skip_on) {
        fwd_launch_s<T, GL, 1>(P, cams, bricks, scales, items, n_items, tf, frag_rgba, frag_key, counters, sch, st);
    } else {
        if constexpr (GL == GATHER_QUAD) {
            if (P.quad_pair) {
                fwd_launch_s<T, GL, 3>(P, cams, bricks, scales, items, n_items, tf, frag_rgba, frag_key, counters,
                                       sch, st);
                return;
            }
        }
        fwd_launch_s<T, GL, 0>(P, cams, bricks, scales, items, n_items, tf, frag_rgba, frag_key, counters, sch, st);
    }
}

// ===========================================================================
// schedules for the persistent launches
// ===========================================================================

__global__ void k_sched_identity(int* sched, int n) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) sched[i] = i;
}

// bucket = brick of a valid item, nbricks for invalid ones (pulled last)
__global__ void k_sched_hist(FrameParams P, const Item* items, int n, int* hist) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    Item it = items[i];
    atomicAdd(hist + (item_ok(it, P) ? it.brick : P.nbricks), 1);
}

__global__ void k_sched_scatter(FrameParams P, const Item* items, int n, const int* offsets, int* cursor,
                                int* sched) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    Item it = items[i];
    int bkt = item_ok(it, P) ? it.brick : P.nbricks;
    int pos = offsets[bkt] + atomicAdd(cursor + bkt, 1);
    if (pos < n) sched[pos] = i;
}

cudaError_t launch_schedule(const FrameParams& P, const Item* items, int n_items, int order, int* hist,
                            int* offsets, int* cursor, unsigned long long* tmp, int* sched, cudaStream_t st) {
    if (n_items == 0) return cudaSuccess;
    unsigned g = (unsigned)((n_items + 255) / 256);
    if (order == 0) {
        k_sched_identity<<<g, 256, 0, st>>>(sched, n_items);
        return cudaGetLastError();
    }
    cudaMemsetAsync(hist, 0, sizeof(int) * (P.nbricks + 1), st);
    cudaMemsetAsync(cursor, 0, sizeof(int) * (P.nbricks + 1), st);
    k_sched_hist<<<g, 256, 0, st>>>(P, items, n_items, hist);
    k_scan<<<1, 1024, 0, st>>>(hist, offsets, P.nbricks + 1, tmp, nullptr);
    k_sched_scatter<<<g, 256, 0, st>>>(P, items, n_items, offsets, cursor, sched);
    return cudaGetLastError();
}

cudaError_t launch_march_fwd(int dtype, int gather, const FrameParams& P, const CamBasis* cams,
                             const BrickDev* bricks, const float* scales, const Item* items, int n_items,
                             const float4* tf, float4* frag_rgba, int* frag_key, Counters* counters,
                             cudaStream_t st, const Schedule* sch) {
    if (n_items == 0) return cudaSuccess;
#define FWD(T)                                                                                                    \
    (gather == GATHER_CELL                                                                                            \
         ? fwd_launch<T, GATHER_CELL>(P, cams, bricks, scales, items, n_items, tf, frag_rgba, frag_key, counters, sch, st) \
     : gather == GATHER_QUAD                                                                                          \
         ? fwd_launch<T, GATHER_QUAD>(P, cams, bricks, scales, items, n_items, tf, frag_rgba, frag_key, counters, sch, st) \
         : fwd_launch<T, GATHER_LINEAR>(P, cams, bricks, scales, items, n_items, tf, frag_rgba, frag_key, counters, sch, \
                                        st))
    switch (dtype) {
        case 0: FWD(float); break;
        case 1: FWD(__half); break;
        case 2: FWD(__nv_bfloat16); break;
        default: FWD(__nv_fp8_e4m3); break;
    }
#undef FWD
    return cudaGetLastError();
}

// ===========================================================================
// iso-surface fragments (DPV_FRAME_ISO)
// ===========================================================================
//
// Each thread tests the sample pairs (j - 1, j) whose later sample j its
// brick owns, evaluating s_{j-1} itself (it lies in the ghost layer), and
// stops at the first pair across which [s >= iso] changes.  The surface
// point sits at fraction f = (iso - s_{j-1}) / (s_j - s_{j-1}) between the
// two samples; its shading uses the gradient of the trilinear interpolant of
// the cell holding it.  Fragment: (shaded rgb, f), key j; the compositor
// keeps the smallest key.

template <typename T, int GL>
__device__ __forceinline__ unsigned long long iso_item(const FrameParams& P, const CamBasis* cams,
                                                       const BrickDev* bricks, const float* scales, const Item& it,
                                                       long long item, const float4* s_tf, float4* frag_rgba,
                                                       int* frag_key) {
    const BrickDev b = bricks[it.brick];
    const CamBasis cam = cams[it.cam];
    const float scale = scales[b.scale_idx];
    const T* data = (const T*)b.data;
    int lx, ly;
    tile_pixel(threadIdx.x, P.tw, lx, ly);
    int px = (it.tile % P.ntx) * P.tw + lx, py = (it.tile / P.ntx) * P.th + ly;
    long long slot = item * P.tp + threadIdx.x;
    unsigned long long nsamp = 0;
    if (px < P.W && py < P.H) {
        MarchState m;
        int key = KEY_EMPTY;
        float4 out = make_float4(0.f, 0.f, 0.f, 0.f);
        if (brick_samples(P, cam, it.cam, b, px, py, m)) {
            const int n = m.j1 - m.j0;
            CornerCache<T, GL> cc;
            SampleWalker wk;
            wk.init(b);
            int ix, iy, iz;
            float fx, fy, fz;
            // the sample before the brick's first one (none before the ray's first)
            int k = m.j0 == 0 ? 0 : -1;
            wk.at(m, k, ix, iy, iz, fx, fy, fz);
            float sp = trilinear<T, GL>(b, data, scale, cc, ix, iy, iz, fx, fy, fz);
            ++nsamp;
            for (++k; k < n; ++k) {
                wk.at(m, k, ix, iy, iz, fx, fy, fz);
                const float s = trilinear<T, GL>(b, data, scale, cc, ix, iy, iz, fx, fy, fz);
                ++nsamp;
                if ((sp >= P.iso) != (s >= P.iso)) {
                    const float f = (P.iso - sp) / (s - sp);
                    // the surface point, at sample index k - 1 + f of the brick
                    const float fk = (float)(k - 1) + f;
                    int c[3];
                    float w[3];
#pragma unroll
                    for (int a = 0; a < 3; ++a) {
                        const float q = fmaf(fk, m.st[a], m.q0[a]);
                        c[a] = min(max(__float2int_rd(q), 0), b.s_n[a] - 2);
                        w[a] = q - (float)c[a];
                    }
                    trilinear<T, GL>(b, data, scale, cc, c[0], c[1], c[2], w[0], w[1], w[2]);
                    // gradient of the interpolant: each component the
                    // bilinear lerp of the cell's edge differences along
                    // that axis; explicit fma / rounded products, so every
                    // gather layout gives the same bits
                    const float* v = cc.v;
                    auto lerp = [](float t, float a, float b2) { return fmaf(t, b2 - a, a); };
                    const float gx = lerp(w[2], lerp(w[1], v[1] - v[0], v[3] - v[2]), lerp(w[1], v[5] - v[4], v[7] - v[6]));
                    const float gy = lerp(w[2], lerp(w[0], v[2] - v[0], v[3] - v[1]), lerp(w[0], v[6] - v[4], v[7] - v[5]));
                    const float gz = lerp(w[1], lerp(w[0], v[4] - v[0], v[5] - v[1]), lerp(w[0], v[6] - v[2], v[7] - v[3]));
                    const float nn = sqrtf(fmaf(gx, gx, fmaf(gy, gy, __fmul_rn(gz, gz))));
                    const float dn =
                        sqrtf(fmaf(m.st[0], m.st[0], fmaf(m.st[1], m.st[1], __fmul_rn(m.st[2], m.st[2]))));
                    float fac = 1.0f;
                    if (nn > 0.0f) {
                        const float dot = fmaf(gx, m.st[0], fmaf(gy, m.st[1], __fmul_rn(gz, m.st[2])));
                        fac = fmaf(0.75f, __fdiv_rn(fabsf(dot), __fmul_rn(nn, dn)), 0.25f);
                    }
                    const TFSample col = tf_lookup(s_tf, P, P.iso);
                    out = make_float4(__fmul_rn(col.v.x, fac), __fmul_rn(col.v.y, fac), __fmul_rn(col.v.z, fac), f);
                    key = m.j0 + k;
                    break;
                }
                sp = s;
            }
        }
        frag_rgba[slot] = out;
        frag_key[slot] = key;
    }
    return nsamp;
}

template <typename T, int GL>
__global__ void __launch_bounds__(256) k_iso_fwd(FrameParams P, const CamBasis* cams, const BrickDev* bricks,
                                                 const float* scales, const Item* items, const float4* tf,
                                                 float4* frag_rgba, int* frag_key, Counters* counters) {
    extern __shared__ float4 s_tf[];
    for (int i = threadIdx.x; i < P.ntf; i += blockDim.x) s_tf[i] = tf[i];
    __syncthreads();
    const Item it = items[blockIdx.x];
    unsigned long long nsamp = 0;
    if (item_ok(it, P)) nsamp = iso_item<T, GL>(P, cams, bricks, scales, it, blockIdx.x, s_tf, frag_rgba, frag_key);
    nsamp = warp_sum_u64(nsamp);
    if ((threadIdx.x & 31) == 0 && nsamp) atomicAdd(&counters->samples_fwd, nsamp);
}

template <typename T, int GL>
static void iso_launch(const FrameParams& P, const CamBasis* cams, const BrickDev* bricks, const float* scales,
                       const Item* items, int n_items, const float4* tf, float4* frag_rgba, int* frag_key,
                       Counters* counters, cudaStream_t st) {
    size_t smem = sizeof(float4) * P.ntf;
    if (smem > 48 * 1024)
        cudaFuncSetAttribute(k_iso_fwd<T, GL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_iso_fwd<T, GL><<<n_items, P.tp, smem, st>>>(P, cams, bricks, scales, items, tf, frag_rgba, frag_key, counters);
}

cudaError_t launch_iso_fwd(int dtype, int gather, const FrameParams& P, const CamBasis* cams,
                           const BrickDev* bricks, const float* scales, const Item* items, int n_items,
                           const float4* tf, float4* frag_rgba, int* frag_key, Counters* counters, cudaStream_t st) {
    if (n_items == 0) return cudaSuccess;
#define ISO(T)                                                                                                   \
    (gather == GATHER_CELL   ? iso_launch<T, GATHER_CELL>(P, cams, bricks, scales, items, n_items, tf, frag_rgba,    \
                                                          frag_key, counters, st)                                 \
     : gather == GATHER_QUAD ? iso_launch<T, GATHER_QUAD>(P, cams, bricks, scales, items, n_items, tf, frag_rgba,    \
                                                          frag_key, counters, st)                                 \
                             : iso_launch<T, GATHER_LINEAR>(P, cams, bricks, scales, items, n_items, tf, frag_rgba, \
                                                            frag_key, counters, st))
    switch (dtype) {
        case 0: ISO(float); break;
        case 1: ISO(__half); break;
        case 2: ISO(__nv_bfloat16); break;
        default: ISO(__nv_fp8_e4m3); break;
    }
#undef ISO
    return cudaGetLastError();
}

// ===========================================================================
// sort-last compositor (forward)
// ===========================================================================

// The pixel's non-empty fragments in ascending key order.  Up to KR are kept
// sorted in registers (insertion with compile-time indices); `n` may exceed
// KR, in which case the caller falls back to selection from memory.
struct SortedFrags {
    int key[KR];
    int slot[KR];
    int n;
};

__device__ __forceinline__ void collect_sorted(const int* frag_key, long long first, int cnt, int tp, int t,
                                               SortedFrags& s) {
#pragma unroll
    for (int i = 0; i < KR; ++i) {
        s.key[i] = KEY_EMPTY;
        s.slot[i] = -1;
    }
    s.n = 0;
    for (int q = 0; q < cnt; ++q) {
        int k = frag_key[(first + q) * tp + t];
        if (k == KEY_EMPTY) continue;
        int ck = k, cs = q;
#pragma unroll
        for (int i = 0; i < KR; ++i) {
            if (ck < s.key[i]) {
                int tk = s.key[i], ts = s.slot[i];
                s.key[i] = ck;
                s.slot[i] = cs;
                ck = tk;
                cs = ts;
            }
        }
        ++s.n;
    }
}

// Fallback for more than KR fragments: the slot of the smallest key > last.
__device__ __forceinline__ int next_slot(const int* frag_key, long long first, int cnt, int tp, int t, int last) {
    int best = KEY_EMPTY, bs = -1;
    for (int q = 0; q < cnt; ++q) {
        int k = frag_key[(first + q) * tp + t];
        if (k != KEY_EMPTY && k > last && k < best) {
            best = k;
            bs = q;
        }
    }
    return bs;
}

__device__ __forceinline__ float pixel_t_enter(const FrameParams& P, const CamBasis& cam, int c, int px, int py) {
    Ray r;
    load_ray(cam, P, c, px, py, r);
    return r.te;
}

__global__ void __launch_bounds__(256) k_composite_fwd(FrameParams P, float inv_spacing, const CamBasis* cams,
                                                       const int* tile_first, const int* tile_count,
                                                       const Item* items, const float4* frag_rgba,
                                                       const int* frag_key, float4* out_rgba, float* out_depth,
                                                       unsigned char* order) {
    int ct = blockIdx.x;
    int ntiles = P.ntx * P.nty;
    int c = ct / ntiles, tile = ct % ntiles;
    int lx, ly;
    tile_pixel(threadIdx.x, P.tw, lx, ly);
    int px = (tile % P.ntx) * P.tw + lx, py = (tile / P.ntx) * P.th + ly;
    if (px >= P.W || py >= P.H) return;
    long long first_item = tile_first[ct];
    int cnt = tile_count[ct];
    if (first_item < 0 || first_item + cnt > P.items_cap) cnt = 0;    // list overflowed: error bit already set
    // fragment slots: P.deep layers per item (1 unless deep fragments)
    const long long first = first_item * P.deep;
    cnt *= P.deep;
    int t = threadIdx.x;
    SortedFrags s;
    collect_sorted(frag_key, first, cnt, P.tp, t, s);
    float C0 = 0.f, C1 = 0.f, C2 = 0.f, A = 0.f;
    int depth_key = KEY_EMPTY;
    long long pix = ((long long)c * P.H + py) * P.W + px;
    unsigned char* ord = order ? order + pix * P.order_stride : nullptr;
    if (s.n <= KR) {
#pragma unroll
        for (int i = 0; i < KR; ++i) {
            if (i < s.n) {
                float4 f = frag_rgba[(first + s.slot[i]) * P.tp + t];
                float w = 1.0f - A;
                C0 = fmaf(w, f.x, C0);
                C1 = fmaf(w, f.y, C1);
                C2 = fmaf(w, f.z, C2);
                A = fmaf(w, f.w, A);
                if (f.w > 0.0f && depth_key == KEY_EMPTY) depth_key = s.key[i];
                if (ord && i < P.order_stride) ord[i] = (unsigned char)items[first_item + s.slot[i] / P.deep].brick;
            }
        }
    } else {
        int last = -1;
        for (int i = 0; i < s.n; ++i) {
            int q = next_slot(frag_key, first, cnt, P.tp, t, last);
            int k = frag_key[(first + q) * P.tp + t];
            last = k;
            float4 f = frag_rgba[(first + q) * P.tp + t];
            float w = 1.0f - A;
            C0 = fmaf(w, f.x, C0);
            C1 = fmaf(w, f.y, C1);
            C2 = fmaf(w, f.z, C2);
            A = fmaf(w, f.w, A);
            if (f.w > 0.0f && depth_key == KEY_EMPTY) depth_key = k;
            if (ord && i < P.order_stride) ord[i] = (unsigned char)items[first_item + q / P.deep].brick;
        }
    }
    if (ord)
        for (int i = s.n; i < P.order_stride; ++i) ord[i] = 0xFF;
    out_rgba[pix] = make_float4(C0, C1, C2, A);
    float depth = __int_as_float(0x7f800000);
    if (depth_key != KEY_EMPTY) {
        float te = pixel_t_enter(P, cams[c], c, px, py);
        depth = te + ((float)depth_key + 0.5f) * P.dt;
    }
    out_depth[pix] = depth;
}

// Depth composite of iso-surface fragments: the nearest (smallest key)
// opaque fragment, its depth t_{key-1} + f dt from the fraction it carries
// in w.  The order image lists the pixel's fragments front to back.
__global__ void __launch_bounds__(256) k_composite_iso(FrameParams P, const CamBasis* cams, const int* tile_first,
                                                       const int* tile_count, const Item* items,
                                                       const float4* frag_rgba, const int* frag_key,
                                                       float4* out_rgba, float* out_depth, unsigned char* order) {
    int ct = blockIdx.x;
    int ntiles = P.ntx * P.nty;
    int c = ct / ntiles, tile = ct % ntiles;
    int lx, ly;
    tile_pixel(threadIdx.x, P.tw, lx, ly);
    int px = (tile % P.ntx) * P.tw + lx, py = (tile / P.ntx) * P.th + ly;
    if (px >= P.W || py >= P.H) return;
    long long first = tile_first[ct];
    int cnt = tile_count[ct];
    if (first < 0 || first + cnt > P.items_cap) cnt = 0;    // list overflowed: error bit already set
    int t = threadIdx.x;
    SortedFrags s;
    collect_sorted(frag_key, first, cnt, P.tp, t, s);
    long long pix = ((long long)c * P.H + py) * P.W + px;
    unsigned char* ord = order ? order + pix * P.order_stride : nullptr;
    int front = -1, front_key = KEY_EMPTY;
    if (s.n <= KR) {
        if (s.n > 0) {
            front = s.slot[0];
            front_key = s.key[0];
        }
        if (ord) {
#pragma unroll
            for (int i = 0; i < KR; ++i)
                if (i < s.n && i < P.order_stride) ord[i] = (unsigned char)items[first + s.slot[i]].brick;
        }
    } else {
        int last = -1;
        for (int i = 0; i < s.n; ++i) {
            int q = next_slot(frag_key, first, cnt, P.tp, t, last);
            int k = frag_key[(first + q) * P.tp + t];
            last = k;
            if (i == 0) {
                front = q;
                front_key = k;
            }
            if (ord && i < P.order_stride) ord[i] = (unsigned char)items[first + q].brick;
        }
    }
    if (ord)
        for (int i = s.n; i < P.order_stride; ++i) ord[i] = 0xFF;
    float4 rgba = make_float4(0.f, 0.f, 0.f, 0.f);
    float depth = __int_as_float(0x7f800000);
    if (front >= 0) {
        const float4 f = frag_rgba[(first + front) * P.tp + t];
        rgba = make_float4(f.x, f.y, f.z, 1.0f);
        const float te = pixel_t_enter(P, cams[c], c, px, py);
        depth = te + ((float)front_key - 0.5f + f.w) * P.dt;
    }
    out_rgba[pix] = rgba;
    out_depth[pix] = depth;
}

cudaError_t launch_composite_iso(const FrameParams& P, const CamBasis* cams, const int* tile_first,
                                 const int* tile_count, const Item* items, const float4* frag_rgba,
                                 const int* frag_key, float4* out_rgba, float* out_depth, unsigned char* order,
                                 cudaStream_t st) {
    int nct = P.ncam * P.ntx * P.nty;
    k_composite_iso<<<nct, P.tp, 0, st>>>(P, cams, tile_first, tile_count, items, frag_rgba, frag_key, out_rgba,
                                          out_depth, order);
    return cudaGetLastError();
}

cudaError_t launch_composite_fwd(const FrameParams& P, float inv_spacing, const CamBasis* cams,
                                 const int* tile_first, const int* tile_count, const Item* items,
                                 const float4* frag_rgba, const int* frag_key, float4* out_rgba, float* out_depth,
                                 unsigned char* order, cudaStream_t st) {
    int nct = P.ncam * P.ntx * P.nty;
    k_composite_fwd<<<nct, P.tp, 0, st>>>(P, inv_spacing, cams, tile_first, tile_count, items, frag_rgba, frag_key,
                                          out_rgba, out_depth, order);
    return cudaGetLastError();
}

// ===========================================================================
// compositor adjoint
// ===========================================================================
//
// For the ordered fragments k = 0..n-1 of a pixel with loss gradient g:
//   T_k   = prod_{m<k} (1 - A_m)                       (transmittance in front)
//   Cb_k, Ab_k = composite of the fragments behind k
//   dL/dC_k = T_k g_rgb
//   dL/dA_k = T_k (g_a (1 - Ab_k) - g_rgb . Cb_k)
__global__ void __launch_bounds__(256) k_composite_bwd(FrameParams P, const int* tile_first, const int* tile_count,
                                                       const float4* frag_rgba, const int* frag_key,
                                                       const float4* grad_img, float4* frag_grad) {
    int ct = blockIdx.x;
    int ntiles = P.ntx * P.nty;
    int c = ct / ntiles, tile = ct % ntiles;
    int lx, ly;
    tile_pixel(threadIdx.x, P.tw, lx, ly);
    int px = (tile % P.ntx) * P.tw + lx, py = (tile / P.ntx) * P.th + ly;
    if (px >= P.W || py >= P.H) return;
    long long first = tile_first[ct];
    int cnt = tile_count[ct];
    if (first < 0 || first + cnt > P.items_cap) cnt = 0;
    int t = threadIdx.x;
    long long pix = ((long long)c * P.H + py) * P.W + px;
    float4 g = grad_img[pix];
    SortedFrags s;
    collect_sorted(frag_key, first, cnt, P.tp, t, s);
    if (s.n <= KR) {
        float Tf[KR];
        float T = 1.0f;
#pragma unroll
        for (int i = 0; i < KR; ++i) {
            Tf[i] = T;
            if (i < s.n) T *= 1.0f - frag_rgba[(first + s.slot[i]) * P.tp + t].w;
        }
        float Cb0 = 0.f, Cb1 = 0.f, Cb2 = 0.f, Ab = 0.f;
#pragma unroll
        for (int i = KR - 1; i >= 0; --i) {
            if (i < s.n) {
                long long o = (first + s.slot[i]) * P.tp + t;
                float4 f = frag_rgba[o];
                float gA = Tf[i] * (g.w * (1.0f - Ab) - (g.x * Cb0 + g.y * Cb1 + g.z * Cb2));
                frag_grad[o] = make_float4(Tf[i] * g.x, Tf[i] * g.y, Tf[i] * g.z, gA);
                float w = 1.0f - f.w;
                Cb0 = fmaf(w, Cb0, f.x);
                Cb1 = fmaf(w, Cb1, f.y);
                Cb2 = fmaf(w, Cb2, f.z);
                Ab = fmaf(w, Ab, f.w);
            }
        }
    } else {
        // more than KR fragments: walk the order from memory twice
        float T = 1.0f;
        int last = -1;
        for (int i = 0; i < s.n; ++i) {          // front to back: store T_k in the grad slot
            int q = next_slot(frag_key, first, cnt, P.tp, t, last);
            long long o = (first + q) * P.tp + t;
            last = frag_key[o];
            frag_grad[o] = make_float4(T, 0.f, 0.f, 0.f);
            T *= 1.0f - frag_rgba[o].w;
        }
        float Cb0 = 0.f, Cb1 = 0.f, Cb2 = 0.f, Ab = 0.f;
        int prev = KEY_EMPTY;
        for (int i = 0; i < s.n; ++i) {          // back to front
            int best = -1, bq = -1;
            for (int q = 0; q < cnt; ++q) {
                int k = frag_key[(first + q) * P.tp + t];
                if (k != KEY_EMPTY && k < prev && k > best) {
                    best = k;
                    bq = q;
                }
            }
            long long o = (first + bq) * P.tp + t;
            prev = best;
            float Tk = frag_grad[o].x;
            float4 f = frag_rgba[o];
            float gA = Tk * (g.w * (1.0f - Ab) - (g.x * Cb0 + g.y * Cb1 + g.z * Cb2));
            frag_grad[o] = make_float4(Tk * g.x, Tk * g.y, Tk * g.z, gA);
            float w = 1.0f - f.w;
            Cb0 = fmaf(w, Cb0, f.x);
            Cb1 = fmaf(w, Cb1, f.y);
            Cb2 = fmaf(w, Cb2, f.z);
            Ab = fmaf(w, Ab, f.w);
        }
    }
}

cudaError_t launch_composite_bwd(const FrameParams& P, const int* tile_first, const int* tile_count,
                                 const float4* frag_rgba, const int* frag_key, const float4* grad_img,
                                 float4* frag_grad, cudaStream_t st) {
    int nct = P.ncam * P.ntx * P.nty;
    k_composite_bwd<<<nct, P.tp, 0, st>>>(P, tile_first, tile_count, frag_rgba, frag_key, grad_img, frag_grad);
    return cudaGetLastError();
}

// ===========================================================================
// ray-march adjoint
// ===========================================================================
//
// Replays the fragment's samples front to back with the forward's exact
// arithmetic (same early-termination decisions), recomputing transmittance
// instead of storing it.  For fragment (C, A) with gradient (gC, gA) and
// sample i (opacity a_i, colour c_i, transmittance T_i):
//   S_i       = C - C_{<=i}                  (what the samples behind add)
//   dC/dc_i   = T_i a_i
//   dC/da_i   = T_i c_i - S_i / (1 - a_i)
//   dA/da_i   = (1 - A) / (1 - a_i)
//   da_i/dsig = dt (1 - a_i),  sigma = sigma_max * alpha_TF
// then the TF lerp (weights 1-w, w on entries i0, i0+1), ds from the lerp
// slope, and the eight trilinear weights scatter into the global field.
//
// Accumulation: consecutive samples of a ray usually fall in the same TF
// segment, so each thread sums its TF gradient in registers while the
// segment stays the same and flushes on change; a step to the neighbouring
// segment keeps the sums of the entry the two segments share.  Nearby rays share TF
// segments, so a single shared table would serialise the flushes of a warp
// on the same addresses; the CTA keeps `ncopy` copies of the TF gradient
// table (bwd_tf_copies; the copy of a lane: tf_copy) (copies offset by one
// float so equal entries of different copies sit in different banks).
// Each copy is a compensated FP32 sum: a high part and a low part per entry
// (tf_add_comp), so that a copy's value does not drift with the number of
// flushes it takes or with how much they cancel.  At the end the copies
// are summed the same way and added to the global FP64 table once per
// touched entry.  The voxel gradient goes, per sample, as two
// float4 reductions into the face adjoint buffer (gather layout; one float4
// per cell face; k_face_gather then writes the field) -- measured 3 % faster
// than summing a cell run in eight registers first -- or, without that
// buffer, as cell runs flushed with eight FP32 atomics into the global field.

struct TFRunF {
    int i0 = -1;
    float a[8];        // entry i0 (rgba), entry i0+1 (rgba)
};

// Knuth's TwoSum: s = fl(a + b) and the exact rounding error e, a + b = s + e.
__device__ __forceinline__ float two_sum_err(float a, float b, float s) {
    float bb = s - a;
    return (a - (s - bb)) + (b - bb);
}

// Compensated shared accumulation of x into the entry at `hi` (the entry's
// low part sits `lo` floats further on).  The atomic returns the value o it
// added x to; the sum it stored is fl(o + x), rounded to nearest like the
// register sum below, so TwoSum recovers the exact rounding error of that
// addition, which goes into the low part.  hi + lo then equals the sum of
// every x up to the rounding of the low part's own sums (errors of errors),
// whatever the order of the flushes and however much they cancel.
__device__ __forceinline__ void tf_add_comp(float* hi, int lo, float x) {
    const float o = atomicAdd(hi, x);
    const float e = two_sum_err(o, x, o + x);
    if (e != 0.0f) atomicAdd(hi + lo, e);
}

__device__ __forceinline__ void tf_flush_f(TFRunF& r, float* tab, int lo) {
    if (r.i0 < 0) return;
    float* e = tab + 4 * r.i0;
#pragma unroll
    for (int c = 0; c < 8; ++c)
        if (r.a[c] != 0.0f) tf_add_comp(e + c, lo, r.a[c]);
}

// Copies of the compensated TF gradient table per CTA (a high and a low
// part per entry): as many as fit in 64 KB of shared memory, at most `cap`.
// Shared memory and L1 share each SM's 256 KB and registers hold the
// kernel to three CTAs per SM either way: at 256 entries a copy takes 8 KB.
// Where the face reductions mostly hit L2 (per-sample reductions), the
// shared-memory atomics bound the replay and more copies pay; where they go
// to DRAM (cell runs), the replay is bound by them and L1 for the gather
// pays.  Measured (replay, 256 entries): 512^3 f32 one camera 2 copies
// 7.86 ms, 4 copies 6.83, 6 copies 6.66, 8 copies 7.01; 512^3 bf16 two
// cameras 12.6, 10.83, 10.57, 10.70 ms; 2048^3 bf16 (cell runs) 1 copy
// 770.8 ms, 2 760.4, 3 751.2, 4 748.4, 6 779.5.  (Plain FP32 copies, one
// part per entry, at 512^3 f32: 16 copies 7.61 ms, 8 copies 6.72, 4 copies
// 6.81, 2 copies 7.16.)
int bwd_tf_copies(int ntf, int cap) {
    int c = 65536 / (32 * ntf);
    return c < 1 ? 1 : (c > cap ? cap : c);
}

// Floats of one copy: high parts, low parts, one float of padding.
__host__ __device__ __forceinline__ int tf_copy_stride(int ntf) { return 8 * ntf + 1; }

// Sum of entry i over the copies (high and low parts), compensated, into
// the global FP64 table.
__device__ __forceinline__ void tf_copies_to_global(const float* s_g, int ncopy, int ntf, int i, double* dtf) {
    const int stride = tf_copy_stride(ntf), lo = 4 * ntf;
    float s = 0.0f, e = 0.0f;
    for (int c = 0; c < ncopy; ++c) {
        const float h = s_g[c * stride + i];
        const float t = s + h;
        e += two_sum_err(s, h, t) + s_g[c * stride + lo + i];
        s = t;
    }
    const double v = (double)s + (double)e;
    if (v != 0.0) atomicAdd(dtf + i, v);
}

// The copy a thread flushes into.  A warp covers an 8 x 4 pixel block (lane
// = x + 8 y), and neighbouring rays tend to hit the same TF entries, so the
// lanes that share a copy lie on a diagonal, (x + 2 y) mod ncopy, rather
// than in one column (x mod ncopy): 6.72 -> 6.54 ms at mid with 8 copies.
__device__ __forceinline__ int tf_copy(int tid, int ncopy) {
    return ((tid & 7) + 2 * ((tid >> 3) & 3)) % ncopy;
}

// Forms of the field gradient (template parameter FACE): 0 scalar atomics
// into the field (cell runs of eight registers); 1 the face buffer, two
// vector reductions per sample; 2 the face buffer, one pair of vector
// reductions per run of samples in one cell.  Per sample is faster where
// the reductions mostly hit L2 (bricks of 257^3: 1.7 % at 512^3); per run
// where they go to DRAM (bricks of 513^3 at 2048^3: 11.6 % faster), since
// a run halves them (about two samples per cell at half-voxel steps).

// The face buffer interleaves pairs of z layers: face (x, y, z) of a brick
// is slot ((z / 2) qxy + y qx + x) 2 + z % 2, so the lower and upper faces
// of a cell at even z share one 32-byte sector (one DRAM read-modify-write
// instead of two where the reductions miss L2).  A brick's slot count is
// even, so a slot's parity is its face's z parity.
__device__ __forceinline__ long long face_slot(const BrickDev& b, int x, int y, int z) {
    return ((long long)(z >> 1) * b.qxy + (long long)y * b.qx + x) * 2 + (z & 1);
}
// The upper face of the cell whose lower face is slot s.
__device__ __forceinline__ long long face_above(long long s, int qxy) {
    return (s & 1) ? s + 2 * (long long)qxy - 1 : s + 1;
}

__device__ __forceinline__ void face_flush(CellRun& r, float4* gface, int qxy) {
    if (r.base < 0) return;
    atomicAdd(gface + r.base, make_float4(r.a[0], r.a[1], r.a[2], r.a[3]));
    atomicAdd(gface + face_above(r.base, qxy), make_float4(r.a[4], r.a[5], r.a[6], r.a[7]));
}

// One work item of the adjoint: replay each thread's fragment and
// accumulate its TF gradient into `my_tab` (a shared copy) and its voxel
// gradient into the global field.  Returns the samples replayed.
template <typename T, int GL, int FACE>
__device__ __forceinline__ unsigned long long bwd_item(const FrameParams& P, const CamBasis* cams,
                                                       const BrickDev* bricks, const float* scales, const Item& it,
                                                       long long item, int t, const float4* s_tf, float* my_tab,
                                                       const float4* frag_rgba, const int* frag_key,
                                                       const float4* frag_grad, float* dvol, float4* gface,
                                                       long long gbase) {
    const BrickDev b = bricks[it.brick];
    const CamBasis cam = cams[it.cam];
    const float scale = scales[b.scale_idx];
    const T* data = (const T*)b.data;
    int lx, ly;
    tile_pixel(t, P.tw, lx, ly);
    int px = (it.tile % P.ntx) * P.tw + lx, py = (it.tile / P.ntx) * P.th + ly;
    long long slot = item * P.tp + t;
    unsigned nsamp = 0;
    const float gscale = Storage<T>::unit_scale ? 1.0f : scale;
    const long long sy = P.dims[0], sz = (long long)P.dims[0] * P.dims[1];
    const int tf_lo = 4 * P.ntf;          // low parts of the copy, after its high parts
    if (px < P.W && py < P.H && frag_key[slot] != KEY_EMPTY) {
        MarchState m;
        float4 F = frag_rgba[slot];
        float4 G = frag_grad[slot];
        if (brick_samples(P, cam, it.cam, b, px, py, m) && (G.x != 0.f || G.y != 0.f || G.z != 0.f || G.w != 0.f)) {
            float C0 = 0.f, C1 = 0.f, C2 = 0.f, Tr = 1.0f;
            const float GwT = G.w * (1.0f - F.w);     // G_a (1 - A): the only use of G_a and A below
            int n = m.j1 - m.j0;
            TFRunF tr;
            CellRun cr;
            const long long gofs = (long long)b.s_lo[2] * sz + (long long)b.s_lo[1] * sy + b.s_lo[0];
            CornerCache<T, GL> cc;
            SampleWalker wk;
            wk.init(b);
            // narrow quad layouts fetch the next sample's faces one sample
            // ahead (their raw vectors take four registers); the
            // interpolation is trilinear()'s, bit for bit
            constexpr bool ahead = GL == GATHER_QUAD && sizeof(T) <= 2;
            GatherRaw<T, GATHER_QUAD> raw;
            int nix = 0, niy = 0, niz = 0;
            float nfx = 0.f, nfy = 0.f, nfz = 0.f;
            if (ahead && n > 0) {
                wk.at(m, 0, nix, niy, niz, nfx, nfy, nfz);
                raw.fetch(b, nix, niy, niz);
            }
            for (int k = 0; k < n; ++k) {
                int ix, iy, iz;
                float fx, fy, fz;
                float s;
                if (ahead) {
                    ix = nix;
                    iy = niy;
                    iz = niz;
                    fx = nfx;
                    fy = nfy;
                    fz = nfz;
                    float v[8];
                    raw.decode(v);
                    if (k + 1 < n) {
                        wk.at(m, k + 1, nix, niy, niz, nfx, nfy, nfz);
                        raw.fetch(b, nix, niy, niz);
                    }
                    s = lerp_cell<T>(v, fx, fy, fz, scale);
                } else {
                    wk.at(m, k, ix, iy, iz, fx, fy, fz);
                    s = trilinear<T, GL>(b, data, scale, cc, ix, iy, iz, fx, fy, fz);
                }
                float4 dsl;
                TFSample c = tf_lookup_slope(s_tf, P, s, dsl);
                float al = sample_alpha(P, c.v.w);
                float ta = Tr * al;
                float n0 = fmaf(ta, c.v.x, C0), n1 = fmaf(ta, c.v.y, C1), n2 = fmaf(ta, c.v.z, C2);
                float om = 1.0f - al;
                // dL/dalpha times dalpha/dsigma = dt (1 - alpha), with (1 - alpha)
                // multiplied into the bracket: no division by 1 - alpha
                //   dL/dsigma = dt (sum_c G_c (T c_c (1 - alpha) - S_c) + G_a (1 - A))
                float S0 = F.x - n0, S1 = F.y - n1, S2 = F.z - n2;
                float Tom = Tr * om;
                float gal = G.x * fmaf(Tom, c.v.x, -S0) + G.y * fmaf(Tom, c.v.y, -S1) + G.z * fmaf(Tom, c.v.z, -S2) +
                            GwT;
                float g_r = G.x * ta, g_g = G.y * ta, g_b = G.z * ta;
                float g_a = gal * P.sdt;
                if (c.i0 != tr.i0) {
                    if (tr.i0 >= 0 && c.i0 == tr.i0 + 1) {
                        // the next segment shares entry i0 + 1: keep its sums
                        float* e = my_tab + 4 * tr.i0;
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            if (tr.a[q] != 0.0f) tf_add_comp(e + q, tf_lo, tr.a[q]);
                            tr.a[q] = tr.a[q + 4];
                            tr.a[q + 4] = 0.0f;
                        }
                    } else if (tr.i0 >= 0 && c.i0 == tr.i0 - 1) {
                        // the previous segment shares entry i0
                        float* e = my_tab + 4 * (tr.i0 + 1);
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            if (tr.a[q + 4] != 0.0f) tf_add_comp(e + q, tf_lo, tr.a[q + 4]);
                            tr.a[q + 4] = tr.a[q];
                            tr.a[q] = 0.0f;
                        }
                    } else {
                        tf_flush_f(tr, my_tab, tf_lo);
#pragma unroll
                        for (int q = 0; q < 8; ++q) tr.a[q] = 0.0f;
                    }
                    tr.i0 = c.i0;
                }
                float w1 = c.w, w0 = 1.0f - c.w;
                tr.a[0] = fmaf(w0, g_r, tr.a[0]);
                tr.a[1] = fmaf(w0, g_g, tr.a[1]);
                tr.a[2] = fmaf(w0, g_b, tr.a[2]);
                tr.a[3] = fmaf(w0, g_a, tr.a[3]);
                tr.a[4] = fmaf(w1, g_r, tr.a[4]);
                tr.a[5] = fmaf(w1, g_g, tr.a[5]);
                tr.a[6] = fmaf(w1, g_b, tr.a[6]);
                tr.a[7] = fmaf(w1, g_a, tr.a[7]);
                if ((FACE || dvol) && c.duds != 0.0f) {
                    float gs = (g_r * dsl.x + g_g * dsl.y + g_b * dsl.z + g_a * dsl.w) * c.duds * gscale;
                    if (FACE == 1 && gs != 0.0f) {
                        // straight into the face buffer, two vector reductions per
                        // sample: cheaper than a register run per cell, whose
                        // eight accumulators cost the loop registers
                        const long long gb = b.gface_off - gbase + face_slot(b, ix, iy, iz);
                        float ax = 1.0f - fx, ay = 1.0f - fy, az = 1.0f - fz;
                        float gyz0 = gs * ay * az, gyz1 = gs * fy * az, gyz2 = gs * ay * fz, gyz3 = gs * fy * fz;
                        atomicAdd(gface + gb, make_float4(gyz0 * ax, gyz0 * fx, gyz1 * ax, gyz1 * fx));
                        atomicAdd(gface + face_above(gb, b.qxy),
                                  make_float4(gyz2 * ax, gyz2 * fx, gyz3 * ax, gyz3 * fx));
                    } else if (FACE == 2 && gs != 0.0f) {
                        // a run per cell: the eight corner sums stay in registers
                        // while the ray stays in the cell, then go to the face
                        // buffer as two vector reductions
                        const long long gb = b.gface_off - gbase + face_slot(b, ix, iy, iz);
                        if (gb != cr.base) {
                            if (cr.base >= 0 && gb == face_above(cr.base, b.qxy)) {
                                // one cell up in z: the old upper face is the new
                                // lower face; only the old lower face leaves
                                atomicAdd(gface + cr.base, make_float4(cr.a[0], cr.a[1], cr.a[2], cr.a[3]));
#pragma unroll
                                for (int q = 0; q < 4; ++q) {
                                    cr.a[q] = cr.a[q + 4];
                                    cr.a[q + 4] = 0.0f;
                                }
                            } else if (cr.base >= 0 && face_above(gb, b.qxy) == cr.base) {
                                // one cell down in z: the old lower face is the new upper face
                                atomicAdd(gface + face_above(cr.base, b.qxy),
                                          make_float4(cr.a[4], cr.a[5], cr.a[6], cr.a[7]));
#pragma unroll
                                for (int q = 0; q < 4; ++q) {
                                    cr.a[q + 4] = cr.a[q];
                                    cr.a[q] = 0.0f;
                                }
                            } else {
                                face_flush(cr, gface, b.qxy);
#pragma unroll
                                for (int q = 0; q < 8; ++q) cr.a[q] = 0.0f;
                            }
                            cr.base = gb;
                        }
                        float ax = 1.0f - fx, ay = 1.0f - fy, az = 1.0f - fz;
                        float gyz0 = gs * ay * az, gyz1 = gs * fy * az, gyz2 = gs * ay * fz, gyz3 = gs * fy * fz;
                        cr.a[0] = fmaf(gyz0, ax, cr.a[0]);
                        cr.a[1] = fmaf(gyz0, fx, cr.a[1]);
                        cr.a[2] = fmaf(gyz1, ax, cr.a[2]);
                        cr.a[3] = fmaf(gyz1, fx, cr.a[3]);
                        cr.a[4] = fmaf(gyz2, ax, cr.a[4]);
                        cr.a[5] = fmaf(gyz2, fx, cr.a[5]);
                        cr.a[6] = fmaf(gyz3, ax, cr.a[6]);
                        cr.a[7] = fmaf(gyz3, fx, cr.a[7]);
                    } else if (!FACE && gs != 0.0f) {
                        long long gb = gofs + (long long)iz * sz + (long long)iy * sy + ix;
                        if (gb != cr.base) {
                            cell_flush(cr, dvol, sy, sz);
                            cr.base = gb;
#pragma unroll
                            for (int q = 0; q < 8; ++q) cr.a[q] = 0.0f;
                        }
                        float ax = 1.0f - fx, ay = 1.0f - fy, az = 1.0f - fz;
                        float gyz0 = gs * ay * az, gyz1 = gs * fy * az, gyz2 = gs * ay * fz, gyz3 = gs * fy * fz;
                        cr.a[0] = fmaf(gyz0, ax, cr.a[0]);
                        cr.a[1] = fmaf(gyz0, fx, cr.a[1]);
                        cr.a[2] = fmaf(gyz1, ax, cr.a[2]);
                        cr.a[3] = fmaf(gyz1, fx, cr.a[3]);
                        cr.a[4] = fmaf(gyz2, ax, cr.a[4]);
                        cr.a[5] = fmaf(gyz2, fx, cr.a[5]);
                        cr.a[6] = fmaf(gyz3, ax, cr.a[6]);
                        cr.a[7] = fmaf(gyz3, fx, cr.a[7]);
                    }
                }
                C0 = n0;
                C1 = n1;
                C2 = n2;
                Tr = Tr - ta;
                if (P.ert_on && 1.0f - Tr > P.ert) {
                    n = k + 1;                          // the samples replayed
                    break;
                }
            }
            nsamp = (unsigned)n;
            tf_flush_f(tr, my_tab, tf_lo);
            if (!FACE && dvol) cell_flush(cr, dvol, sy, sz);
            if (FACE == 2) face_flush(cr, gface, b.qxy);
        }
    }
    return nsamp;
}

template <typename T, int GL, int FACE>
__global__ void __launch_bounds__(256, 3) k_march_bwd(FrameParams P, const CamBasis* cams, const BrickDev* bricks,
                                                   const float* scales, const Item* items, const float4* tf,
                                                   const float4* frag_rgba, const int* frag_key,
                                                   const float4* frag_grad, int ncopy, double* dtf, float* dvol,
                                                   float4* gface, FaceGroup fg, Counters* counters) {
    extern __shared__ float4 s_mem[];
    const Item it = items[blockIdx.x];
    // an item of a brick outside the face group: the whole CTA leaves
    if (FACE && (it.brick < fg.k0 || it.brick >= fg.k1)) return;
    float4* s_tf = s_mem;
    float* s_g = (float*)(s_mem + P.ntf);
    const int stride = tf_copy_stride(P.ntf);
    for (int i = threadIdx.x; i < P.ntf; i += blockDim.x) s_tf[i] = tf[i];
    for (int i = threadIdx.x; i < ncopy * stride; i += blockDim.x) s_g[i] = 0.0f;
    __syncthreads();
    float* my_tab = s_g + tf_copy(threadIdx.x, ncopy) * stride;
    unsigned long long nsamp = 0;
    if (item_ok(it, P))
        nsamp = bwd_item<T, GL, FACE>(P, cams, bricks, scales, it, blockIdx.x, threadIdx.x, s_tf, my_tab, frag_rgba,
                                      frag_key, frag_grad, dvol, gface, fg.base);
    nsamp = warp_sum_u64(nsamp);
    if ((threadIdx.x & 31) == 0 && nsamp) atomicAdd(&counters->samples_bwd, nsamp);
    __syncthreads();
    for (int i = threadIdx.x; i < 4 * P.ntf; i += blockDim.x) tf_copies_to_global(s_g, ncopy, P.ntf, i, dtf);
}

// Persistent adjoint: each warp pulls one warp's share of a work item (32
// pixels of its tile) at a time, in schedule order; a warp whose rays are
// short takes the next unit at once, with no barrier between units.  Each
// CTA's TF tables are added to the global table once, after its warps have
// run out of units.
template <typename T, int GL, int FACE>
__global__ void __launch_bounds__(256, 3) k_march_bwd_persistent(FrameParams P, const CamBasis* cams,
                                                              const BrickDev* bricks, const float* scales,
                                                              const Item* items, const int* sched, int n_items,
                                                              unsigned int* work, const float4* tf,
                                                              const float4* frag_rgba, const int* frag_key,
                                                              const float4* frag_grad, int ncopy, double* dtf,
                                                              float* dvol, float4* gface, FaceGroup fg,
                                                              Counters* counters) {
    extern __shared__ float4 s_mem[];
    float4* s_tf = s_mem;
    float* s_g = (float*)(s_mem + P.ntf);
    const int stride = tf_copy_stride(P.ntf);
    for (int i = threadIdx.x; i < P.ntf; i += blockDim.x) s_tf[i] = tf[i];
    for (int i = threadIdx.x; i < ncopy * stride; i += blockDim.x) s_g[i] = 0.0f;
    __syncthreads();
    float* my_tab = s_g + tf_copy(threadIdx.x, ncopy) * stride;
    const int lane = threadIdx.x & 31;
    const unsigned wpt = (unsigned)(P.tp >> 5);               // warps per tile
    const unsigned n_units = (unsigned)n_items * wpt;
    unsigned long long nsamp = 0;
    for (;;) {
        __syncwarp();
        unsigned u = 0;
        if (lane == 0) u = atomicAdd(work, 1u);
        u = __shfl_sync(0xffffffffu, u, 0);
        if (u >= n_units) break;
        const int item = sched[u / wpt];
        const Item it = items[item];
        if (item_ok(it, P) && (!FACE || (it.brick >= fg.k0 && it.brick < fg.k1)))
            nsamp += bwd_item<T, GL, FACE>(P, cams, bricks, scales, it, item, (int)((u % wpt) * 32 + lane), s_tf,
                                           my_tab, frag_rgba, frag_key, frag_grad, dvol, gface, fg.base);
    }
    nsamp = warp_sum_u64(nsamp);
    if (lane == 0 && nsamp) atomicAdd(&counters->samples_bwd, nsamp);
    __syncthreads();
    for (int i = threadIdx.x; i < 4 * P.ntf; i += blockDim.x) tf_copies_to_global(s_g, ncopy, P.ntf, i, dtf);
}

template <typename T, int GL, int FACE>
static void bwd_launch_f(const FrameParams& P, const CamBasis* cams, const BrickDev* bricks, const float* scales,
                         const Item* items, int n_items, const float4* tf, const float4* frag_rgba,
                         const int* frag_key, const float4* frag_grad, double* dtf, float* dvol, float4* gface,
                         FaceGroup fg, Counters* counters, const Schedule* sch, cudaStream_t st) {
    int ncopy = bwd_tf_copies(P.ntf, FACE == 1 ? 6 : 4);
    size_t smem = sizeof(float4) * P.ntf + sizeof(float) * (size_t)ncopy * tf_copy_stride(P.ntf);
    if (sch) {
        if (smem > 48 * 1024)
            cudaFuncSetAttribute(k_march_bwd_persistent<T, GL, FACE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem);
        int per_sm = 0, dev = 0, nsm = 148;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_march_bwd_persistent<T, GL, FACE>, P.tp, smem);
        int grid = nsm * (per_sm > 0 ? per_sm : 1);
        if (grid > n_items) grid = n_items;
        cudaMemsetAsync(sch->work, 0, sizeof(unsigned int), st);
        k_march_bwd_persistent<T, GL, FACE><<<grid, P.tp, smem, st>>>(P, cams, bricks, scales, items, sch->sched,
                                                                  n_items, sch->work, tf, frag_rgba, frag_key,
                                                                  frag_grad, ncopy, dtf, dvol, gface, fg, counters);
        return;
    }
    if (smem > 48 * 1024)
        cudaFuncSetAttribute(k_march_bwd<T, GL, FACE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_march_bwd<T, GL, FACE><<<n_items, P.tp, smem, st>>>(P, cams, bricks, scales, items, tf, frag_rgba, frag_key,
                                                            frag_grad, ncopy, dtf, dvol, gface, fg, counters);
}

// the face-buffer path and the scalar-atomic path are separate instances
template <typename T, int GL>
static void bwd_launch(const FrameParams& P, const CamBasis* cams, const BrickDev* bricks, const float* scales,
                       const Item* items, int n_items, const float4* tf, const float4* frag_rgba, const int* frag_key,
                       const float4* frag_grad, double* dtf, float* dvol, float4* gface, FaceGroup fg,
                       Counters* counters, const Schedule* sch, cudaStream_t st) {
    if (gface && fg.runs)
        bwd_launch_f<T, GL, 2>(P, cams, bricks, scales, items, n_items, tf, frag_rgba, frag_key, frag_grad, dtf, dvol,
                               gface, fg, counters, sch, st);
    else if (gface)
        bwd_launch_f<T, GL, 1>(P, cams, bricks, scales, items, n_items, tf, frag_rgba, frag_key, frag_grad, dtf, dvol,
                               gface, fg, counters, sch, st);
    else
        bwd_launch_f<T, GL, 0>(P, cams, bricks, scales, items, n_items, tf, frag_rgba, frag_key, frag_grad, dtf, dvol,
                               gface, fg, counters, sch, st);
}

cudaError_t launch_march_bwd(int dtype, int gather, const FrameParams& P, const CamBasis* cams,
                             const BrickDev* bricks, const float* scales, const Item* items, int n_items,
                             const float4* tf, const float4* frag_rgba, const int* frag_key,
                             const float4* frag_grad, double* dtf, float* dvol, float4* gface,
                             Counters* counters, cudaStream_t st, const Schedule* sch, const FaceGroup* fgp) {
    if (n_items == 0) return cudaSuccess;
    const FaceGroup fg = fgp ? *fgp : FaceGroup{0, P.nbricks, 0, 0};
#define BWD(T)                                                                                                  \
    (gather == GATHER_CELL                                                                                          \
         ? bwd_launch<T, GATHER_CELL>(P, cams, bricks, scales, items, n_items, tf, frag_rgba, frag_key, frag_grad,   \
                                      dtf, dvol, gface, fg, counters, sch, st)                                      \
     : gather == GATHER_QUAD                                                                                        \
         ? bwd_launch<T, GATHER_QUAD>(P, cams, bricks, scales, items, n_items, tf, frag_rgba, frag_key, frag_grad,   \
                                      dtf, dvol, gface, fg, counters, sch, st)                                      \
         : bwd_launch<T, GATHER_LINEAR>(P, cams, bricks, scales, items, n_items, tf, frag_rgba, frag_key, frag_grad, \
                                        dtf, dvol, gface, fg, counters, sch, st))
    switch (dtype) {
        case 0: BWD(float); break;
        case 1: BWD(__half); break;
        case 2: BWD(__nv_bfloat16); break;
        default: BWD(__nv_fp8_e4m3); break;
    }
#undef BWD
    return cudaGetLastError();
}

// ===========================================================================
// gather layout (quad): per cell face the 2 x 2 corners in one vector
// ===========================================================================

template <typename T>
__global__ void k_build_quad(const T* src, int sx, int sy, int sz, typename Quad<T>::W* dst) {
    using W = typename Quad<T>::W;
    long long qx = sx - 1, qxy = (long long)(sx - 1) * (sy - 1);
    long long n = qxy * sz;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        long long z = i / qxy, r = i - z * qxy, y = r / qx, x = r - y * qx;
        long long o = (z * sy + y) * sx + x;
        // interleaved pairs of z layers (quad_slot)
        const long long slot = ((z >> 1) * qxy + r) * 2 + (z & 1);
        W w;
        if constexpr (sizeof(T) == 4) {
            const float* f = (const float*)src;
            w = make_float4(f[o], f[o + 1], f[o + sx], f[o + sx + 1]);
        } else if constexpr (sizeof(T) == 2) {
            const unsigned short* h = (const unsigned short*)src;
            w = make_uint2((unsigned)h[o] | ((unsigned)h[o + 1] << 16), (unsigned)h[o + sx] | ((unsigned)h[o + sx + 1] << 16));
        } else {
            const unsigned char* c = (const unsigned char*)src;
            w = (unsigned)c[o] | ((unsigned)c[o + 1] << 8) | ((unsigned)c[o + sx] << 16) | ((unsigned)c[o + sx + 1] << 24);
        }
        dst[slot] = w;
    }
}

size_t quad_bytes(int dtype, const int s_n[3]) {
    size_t cells = (size_t)(s_n[0] - 1) * (s_n[1] - 1) * (s_n[2] + (s_n[2] & 1));   // z padded to pairs
    static const size_t w[4] = {16, 8, 8, 4};
    return cells * w[dtype];
}

cudaError_t launch_build_quad(int dtype, const void* src, const int s_n[3], void* dst, cudaStream_t st) {
    long long n = (long long)(s_n[0] - 1) * (s_n[1] - 1) * s_n[2];
    long long nb = (n + 255) / 256;
    int blocks = (int)(nb < 148LL * 32 ? nb : 148LL * 32);
    switch (dtype) {
        case 0: k_build_quad<float><<<blocks, 256, 0, st>>>((const float*)src, s_n[0], s_n[1], s_n[2], (float4*)dst); break;
        case 1: k_build_quad<__half><<<blocks, 256, 0, st>>>((const __half*)src, s_n[0], s_n[1], s_n[2], (uint2*)dst); break;
        case 2: k_build_quad<__nv_bfloat16><<<blocks, 256, 0, st>>>((const __nv_bfloat16*)src, s_n[0], s_n[1], s_n[2], (uint2*)dst); break;
        default: k_build_quad<__nv_fp8_e4m3><<<blocks, 256, 0, st>>>((const __nv_fp8_e4m3*)src, s_n[0], s_n[1], s_n[2], (unsigned*)dst); break;
    }
    return cudaGetLastError();
}

// ===========================================================================
// gather layout (cell): per cell its eight corners in one vector
// ===========================================================================

template <typename T>
__global__ void k_build_cell(const T* src, int sx, int sy, int sz, void* dst) {
    const long long cx = sx - 1, cxy = (long long)(sx - 1) * (sy - 1);
    const long long n = cxy * (sz - 1);
    const long long sxy = (long long)sx * sy;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const long long z = i / cxy, r = i - z * cxy, y = r / cx, x = r - y * cx;
        const long long o = (z * sy + y) * sx + x;
        const long long c[8] = {o, o + 1, o + sx, o + sx + 1, o + sxy, o + sxy + 1, o + sxy + sx, o + sxy + sx + 1};
        if constexpr (sizeof(T) == 4) {
            const float* f = (const float*)src;
            float4* d = (float4*)dst + 2 * i;
            d[0] = make_float4(f[c[0]], f[c[1]], f[c[2]], f[c[3]]);
            d[1] = make_float4(f[c[4]], f[c[5]], f[c[6]], f[c[7]]);
        } else if constexpr (sizeof(T) == 2) {
            const unsigned short* h = (const unsigned short*)src;
            unsigned u[4];
            for (int k = 0; k < 4; ++k) u[k] = (unsigned)h[c[2 * k]] | ((unsigned)h[c[2 * k + 1]] << 16);
            ((uint4*)dst)[i] = make_uint4(u[0], u[1], u[2], u[3]);
        } else {
            const unsigned char* b = (const unsigned char*)src;
            unsigned lo = 0, hi = 0;
            for (int k = 0; k < 4; ++k) {
                lo |= (unsigned)b[c[k]] << (8 * k);
                hi |= (unsigned)b[c[4 + k]] << (8 * k);
            }
            ((uint2*)dst)[i] = make_uint2(lo, hi);
        }
    }
}

size_t cell_bytes(int dtype, const int s_n[3]) {
    size_t cells = (size_t)(s_n[0] - 1) * (s_n[1] - 1) * (s_n[2] - 1);
    static const size_t w[4] = {32, 16, 16, 8};
    return cells * w[dtype];
}

cudaError_t launch_build_cell(int dtype, const void* src, const int s_n[3], void* dst, cudaStream_t st) {
    long long n = (long long)(s_n[0] - 1) * (s_n[1] - 1) * (s_n[2] - 1);
    long long nb = (n + 255) / 256;
    int blocks = (int)(nb < 65536 ? nb : 65536);
    if (blocks < 1) return cudaSuccess;
    switch (dtype) {
        case 0: k_build_cell<float><<<blocks, 256, 0, st>>>((const float*)src, s_n[0], s_n[1], s_n[2], dst); break;
        case 1: k_build_cell<__half><<<blocks, 256, 0, st>>>((const __half*)src, s_n[0], s_n[1], s_n[2], dst); break;
        case 2: k_build_cell<__nv_bfloat16><<<blocks, 256, 0, st>>>((const __nv_bfloat16*)src, s_n[0], s_n[1], s_n[2], dst); break;
        default: k_build_cell<__nv_fp8_e4m3><<<blocks, 256, 0, st>>>((const __nv_fp8_e4m3*)src, s_n[0], s_n[1], s_n[2], dst); break;
    }
    return cudaGetLastError();
}

// ===========================================================================
// empty-space skipping: macro-cell value ranges and their transparency
// ===========================================================================
//
// A macro-cell covers 2^MACRO_SHIFT cells per axis of a brick's stored
// region.  Its range [min, max] of decoded node values bounds every sample
// inside (the interpolant is a convex combination, and rounding is
// monotone; so is the product with the brick's scale and the TF coordinate
// u).  The samples then only read TF entries i0(min) .. i0(max) + 1, and if
// all of those have opacity 0 each sample's alpha is exactly 0: skipping it
// leaves the colour and transmittance bit for bit as they are.

size_t macro_cells(const int s_n[3]) {
    size_t m = 1;
    for (int a = 0; a < 3; ++a) m *= (size_t)(((s_n[a] - 2) >> MACRO_SHIFT) + 1);
    return m;
}

template <typename T>
__global__ void k_build_minmax(const T* data, int sx, int sy, int sz, int mx, int my, int mz, float2* mm) {
    const long long n = (long long)mx * my * mz;
    const long long sxy = (long long)sx * sy;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int z = (int)(i / ((long long)mx * my)), r = (int)(i - (long long)z * mx * my), y = r / mx, x = r - y * mx;
        const int x0 = x << MACRO_SHIFT, y0 = y << MACRO_SHIFT, z0 = z << MACRO_SHIFT;
        const int x1 = min(x0 + (1 << MACRO_SHIFT), sx - 1), y1 = min(y0 + (1 << MACRO_SHIFT), sy - 1),
                  z1 = min(z0 + (1 << MACRO_SHIFT), sz - 1);
        float lo = __int_as_float(0x7f800000), hi = -lo;
        for (int zz = z0; zz <= z1; ++zz)
            for (int yy = y0; yy <= y1; ++yy)
                for (int xx = x0; xx <= x1; ++xx) {
                    const float v = Storage<T>::load(data, (int)(zz * sxy + (long long)yy * sx + xx));
                    lo = fminf(lo, v);
                    hi = fmaxf(hi, v);
                }
        mm[i] = make_float2(lo, hi);
    }
}

cudaError_t launch_build_minmax(int dtype, const void* data, const int s_n[3], float2* mm, cudaStream_t st) {
    const int mx = ((s_n[0] - 2) >> MACRO_SHIFT) + 1, my = ((s_n[1] - 2) >> MACRO_SHIFT) + 1,
              mz = ((s_n[2] - 2) >> MACRO_SHIFT) + 1;
    const long long n = (long long)mx * my * mz;
    const int blocks = (int)std::min<long long>((n + 255) / 256, 148LL * 16);
    switch (dtype) {
        case 0: k_build_minmax<float><<<blocks, 256, 0, st>>>((const float*)data, s_n[0], s_n[1], s_n[2], mx, my, mz, mm); break;
        case 1: k_build_minmax<__half><<<blocks, 256, 0, st>>>((const __half*)data, s_n[0], s_n[1], s_n[2], mx, my, mz, mm); break;
        case 2: k_build_minmax<__nv_bfloat16><<<blocks, 256, 0, st>>>((const __nv_bfloat16*)data, s_n[0], s_n[1], s_n[2], mx, my, mz, mm); break;
        default: k_build_minmax<__nv_fp8_e4m3><<<blocks, 256, 0, st>>>((const __nv_fp8_e4m3*)data, s_n[0], s_n[1], s_n[2], mx, my, mz, mm); break;
    }
    return cudaGetLastError();
}

// Z[i] = number of TF entries j <= i with non-zero opacity (one block).
__global__ void k_tf_opaque_prefix(const float4* tf, int n, int* z) {
    __shared__ int s[1024];
    __shared__ int carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int base = 0; base < n; base += blockDim.x) {
        const int i = base + threadIdx.x;
        s[threadIdx.x] = (i < n && tf[i].w != 0.0f) ? 1 : 0;
        __syncthreads();
        for (int o = 1; o < (int)blockDim.x; o <<= 1) {
            const int v = threadIdx.x >= o ? s[threadIdx.x - o] : 0;
            __syncthreads();
            s[threadIdx.x] += v;
            __syncthreads();
        }
        if (i < n) z[i] = carry + s[threadIdx.x];
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) carry += s[threadIdx.x];
        __syncthreads();
    }
}

// TF entry i0 of tf_lookup for value s (same FP32 steps).
__device__ __forceinline__ int tf_entry(const FrameParams& P, float s) {
    float u = fmaf(s, P.tf_scale, P.tf_bias);
    u = fminf(fmaxf(u, 0.0f), (float)(P.ntf - 1));
    return min(__float2int_rd(u), P.ntf - 2);
}

__global__ void k_classify_empty(FrameParams P, const BrickDev* bricks, const float* scales, int unit_scale,
                                 const int* z) {
    const BrickDev b = bricks[blockIdx.y];
    const float scale = scales[b.scale_idx];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < b.mn; i += gridDim.x * blockDim.x) {
        const float2 r = b.mm[i];
        // the samples' values lie in [r.x scale, r.y scale], rounded as the
        // march rounds them (f32 storage is not scaled)
        const float lo = unit_scale ? r.x : r.x * scale, hi = unit_scale ? r.y : r.y * scale;
        const int e0 = tf_entry(P, lo), e1 = tf_entry(P, hi) + 1;
        const int opaque = z[e1] - (e0 > 0 ? z[e0 - 1] : 0);
        b.empty[i] = opaque == 0 ? 1 : 0;
    }
}

cudaError_t launch_classify_empty(int dtype, const FrameParams& P, const BrickDev* bricks, int nbricks,
                                  const float* scales, int max_macro, const float4* tf, int* z, cudaStream_t st) {
    if (nbricks <= 0 || max_macro <= 0) return cudaSuccess;
    k_tf_opaque_prefix<<<1, 1024, 0, st>>>(tf, P.ntf, z);
    const int bx = std::min((max_macro + 255) / 256, 1024);
    k_classify_empty<<<dim3(bx, nbricks), 256, 0, st>>>(P, bricks, scales, dtype == 0 ? 1 : 0, z);
    return cudaGetLastError();
}

// ===========================================================================
// face adjoint buffer -> global field gradient
// ===========================================================================
//
// Node (x, y, z) of a brick is corner (0,0) of face (x, y), corner (1,0) of
// face (x-1, y), corner (0,1) of face (x, y-1) and corner (1,1) of face
// (x-1, y-1) in layer z, where those faces exist.  A global node's gradient
// is the sum of those slots over every brick storing a copy of it (its owner
// and the bricks whose ghost layer holds it), added in neighbour-list order.

size_t face_slots(const int s_n[3]) { return (size_t)(s_n[0] - 1) * (s_n[1] - 1) * (s_n[2] + (s_n[2] & 1)); }

// Rows of nodes a thread gathers at once (face rows ly - 1 .. ly + GR - 1
// are loaded together, each once, so their latencies overlap).
constexpr int GR = 2;

// A thread takes one x column of GR node rows in both layers of a pair of z
// layers (2p, 2p + 1): their face slots are adjacent in the buffer, so each
// of its loads uses the whole 32-byte sector it brings in.
__global__ void __launch_bounds__(128) k_face_gather(const BrickDev* bricks, const int* nb_first, const int* nb,
                                                     const float4* gface, int dims0, int dims1, float* dvol,
                                                     FaceGroup fg, int add) {
    const int o = blockIdx.y;
    const int j0 = nb_first[o], j1 = nb_first[o + 1];
    // with a group: the owner's own slots count if it is in the group; an
    // owner outside it gathers only where a group brick stores its nodes
    const bool own = o >= fg.k0 && o < fg.k1;
    if (!own) {
        bool any = false;
        for (int j = j0 + 1; j < j1; ++j) any = any || (nb[j] >= fg.k0 && nb[j] < fg.k1);
        if (!any) return;
    }
    const BrickDev bo = bricks[o];
    const int nx = bo.o_hi[0] - bo.o_lo[0], ny = bo.o_hi[1] - bo.o_lo[1], nz = bo.o_hi[2] - bo.o_lo[2];
    const int ngy = (ny + GR - 1) / GR;
    // local z of the owned layers: lz0 .. lz0 + nz - 1, spanning the layer
    // pairs p0 .. p0 + npairs - 1 (a pair's layer outside them is skipped;
    // its slots are in the brick's range, the slot count being even)
    const int lz0 = bo.o_lo[2] - bo.s_lo[2];
    const int p0 = lz0 >> 1, npairs = ((lz0 + nz - 1) >> 1) - p0 + 1;
    const int ngroups = ngy * npairs;
    // row groups fastest: neighbouring groups share a face row, which the
    // second one then finds in L2
    for (int grp = blockIdx.x; grp < ngroups; grp += gridDim.x) {
        const int p = p0 + grp / ngy, yy0 = (grp % ngy) * GR;
        const int gy0 = bo.o_lo[1] + yy0;
        const int ly0 = gy0 - bo.s_lo[1];
        // slot of face (0, 0, 2p): face (x, y, 2p + h) is at fo + 2 (y qx + x) + h
        const long long fo = bo.gface_off - fg.base + face_slot(bo, 0, 0, 2 * p);   // read only if own
        // block-uniform trip count
        for (int x0 = 0; x0 < nx; x0 += blockDim.x) {
            const int xo = x0 + threadIdx.x;
            const bool act = xo < nx;
            const int gx = bo.o_lo[0] + xo, lx = gx - bo.s_lo[0];
            const bool xl = lx >= 1, xr = lx <= bo.s_n[0] - 2;
            // face rows ly0 - 1 + k, k = 0 .. GR, both layers: this node's
            // face A and the face to its left (loaded by this thread too: the
            // left neighbour's load brings the line into L1)
            float4 A[GR + 1][2];
            float Ly[GR + 1][2], Lw[GR + 1][2];
#pragma unroll
            for (int k = 0; k <= GR; ++k) {
                const int fy = ly0 - 1 + k;
                const bool row = own && act && fy >= 0 && fy <= bo.s_n[1] - 2 && yy0 - 1 + k < ny;
                const float4* f = gface + fo + 2 * ((long long)fy * bo.qx + lx);
                const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    A[k][h] = row && xr ? f[h] : z4;
                    const float4 q = row && xl ? f[h - 2] : z4;
                    Ly[k][h] = q.y;
                    Lw[k][h] = q.w;
                }
            }
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int zz = 2 * p + h - lz0;
                if (zz < 0 || zz >= nz) continue;
                const int gz = bo.o_lo[2] + zz;
#pragma unroll
                for (int k = 0; k < GR; ++k) {
                    const int yy = yy0 + k;
                    if (!act || yy >= ny) continue;
                    const int gy = gy0 + k;
                    // node row ly0 + k: corner (0,0) of face row k+1, (1,0) of its
                    // left face, (0,1) of face row k, (1,1) of its left face
                    float v = A[k + 1][h].x + Ly[k + 1][h] + A[k][h].z + Lw[k][h];
                    // ghost copies in other bricks exist only for nodes on the
                    // owned box's surface
                    const bool surface =
                        yy == 0 || yy == ny - 1 || zz == 0 || zz == nz - 1 || xo == 0 || xo == nx - 1;
                    if (!own && !surface) continue;
                    // the first pass to reach the node stores it, later passes
                    // add: groups are consecutive rank ranges taken in order,
                    // so the first is the group of the lowest rank storing it
                    bool first = o >= fg.k0;
                    if (surface) {
                        for (int j = j0 + 1; j < j1; ++j) {
                            if (nb[j] >= fg.k1) continue;
                            const BrickDev& b = bricks[nb[j]];
                            const int mx = gx - b.s_lo[0], my = gy - b.s_lo[1], mz = gz - b.s_lo[2];
                            if (mx < 0 || my < 0 || mz < 0 || mx >= b.s_n[0] || my >= b.s_n[1] || mz >= b.s_n[2])
                                continue;
                            if (nb[j] < fg.k0) {
                                first = false;          // an earlier group stores it too
                                continue;
                            }
                            const float4* G = gface + (b.gface_off - fg.base) + face_slot(b, 0, 0, mz);
                            const bool bxl = mx >= 1, bxr = mx <= b.s_n[0] - 2, byl = my >= 1, byr = my <= b.s_n[1] - 2;
                            const long long q0 = 2 * ((long long)my * b.qx + mx), q1 = q0 - 2 * (long long)b.qx;
                            if (bxr && byr) v += G[q0].x;
                            if (bxl && byr) v += G[q0 - 2].y;
                            if (bxr && byl) v += G[q1].z;
                            if (bxl && byl) v += G[q1 - 2].w;
                        }
                    }
                    float* dst = dvol + ((long long)gz * dims1 + gy) * dims0 + gx;
                    if (add && !first)
                        *dst += v;
                    else
                        *dst = v;
                }
            }
        }
    }
}

cudaError_t launch_face_gather(const BrickDev* bricks, int nbricks, const int* nb_first, const int* nb,
                               long long max_rows, const float4* gface, const int dims[3], float* dvol,
                               cudaStream_t st, const FaceGroup* fgp) {
    if (nbricks <= 0 || max_rows <= 0) return cudaSuccess;
    const FaceGroup fg = fgp ? *fgp : FaceGroup{0, nbricks, 0, 0};
    long long groups = (max_rows + GR - 1) / GR;
    long long bx = groups < 4096 ? groups : 4096;
    dim3 grid((unsigned)bx, (unsigned)nbricks);
    k_face_gather<<<grid, 128, 0, st>>>(bricks, nb_first, nb, gface, dims[0], dims[1], dvol, fg, fgp ? 1 : 0);
    return cudaGetLastError();
}

// ===========================================================================
// debug: scatter one rank's fragments into a full frame
// ===========================================================================

__global__ void k_fill_key(int* key, long long n) {
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i < n) key[i] = KEY_EMPTY;
}

__global__ void k_read_frags(FrameParams P, const Item* items, int n_items, int cam, int rank, int layer,
                             const float4* frag_rgba, const int* frag_key, float4* out_rgba, int* out_key) {
    int i = blockIdx.x;
    if (i >= n_items) return;
    Item it = items[i];
    if (!item_ok(it, P) || it.cam != cam || it.brick != rank) return;
    int lx, ly;
    tile_pixel(threadIdx.x, P.tw, lx, ly);
    int px = (it.tile % P.ntx) * P.tw + lx, py = (it.tile / P.ntx) * P.th + ly;
    if (px >= P.W || py >= P.H) return;
    long long slot = ((long long)i * P.deep + layer) * P.tp + threadIdx.x;
    long long pix = (long long)py * P.W + px;
    int k = frag_key[slot];
    out_key[pix] = k;
    out_rgba[pix] = k == KEY_EMPTY ? make_float4(0.f, 0.f, 0.f, 0.f) : frag_rgba[slot];
}

cudaError_t launch_read_frags(const FrameParams& P, const Item* items, int n_items, int cam, int rank, int layer,
                              const float4* frag_rgba, const int* frag_key, float4* out_rgba, int* out_key,
                              cudaStream_t st) {
    long long n = (long long)P.W * P.H;
    cudaMemsetAsync(out_rgba, 0, sizeof(float4) * n, st);
    k_fill_key<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(out_key, n);
    if (n_items)
        k_read_frags<<<n_items, P.tp, 0, st>>>(P, items, n_items, cam, rank, layer, frag_rgba, frag_key, out_rgba,
                                               out_key);
    return cudaGetLastError();
}

}  // namespace dpv
