// dpv_internal.cuh -- device-side data layout and per-sample arithmetic of
// the brick ray-march and the sort-last compositor (sm_103a).
//
// Conventions are the ones stated in include/dpv.h.  Everything here is
// FP32 with integer sample indices; nothing is shared with the FP64 oracle.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace dpv {

constexpr int KEY_EMPTY = 0x7fffffff;
constexpr int MAX_RANKS = 255;
constexpr int MAX_TF = 4096;
constexpr int KR = 16;                   // fragments a pixel sorts in registers
constexpr int RAY_VECS = 5;              // float4 per ray in the ray buffer (see k_rays)

// device error bits (Counters::err)
constexpr unsigned ERR_ITEM_OVERFLOW = 1u;     // culling listed more items than sized for
constexpr unsigned ERR_STAGE_OUTSIDE = 2u;     // a staged sample fell outside its slab box (clamped)
constexpr unsigned ERR_STAGE_INCOMPLETE = 4u;  // a staged ray ended with unmarched samples

// One camera, prepared on the device: eye in node coordinates and the
// orthonormal look-at basis (world directions are node directions up to the
// uniform scale 1/spacing).
struct CamBasis {
    float o[3];
    float f[3], r[3], u[3];
    float th;          // tan(fovy / 2)
    float pad;
};

// Gather layouts of the brick ray-march (template parameter G).
constexpr int GATHER_LINEAR = 0;   // the stored nodes, eight scalar loads
constexpr int GATHER_QUAD = 1;     // two face vectors per sample
constexpr int GATHER_CELL = 2;     // one cell vector per sample

// A value held as the unevaluated sum hi + lo of two floats, |lo| <= ulp(hi)/2:
// about 48 significant bits at FP32 speed (FP64 runs at a small fraction of
// the FP32 rate on this GPU).
struct DF {
    float hi, lo;
};

// Per camera in double-float, rounded once from FP64: eye in node
// coordinates, basis, the pixel scale k = tan(fovy / 2) / H (screen
// x = (2 px + 1 - W) k, y = (2 py + 1 - H) k) and 1 / spacing.
struct CamBasisDF {
    DF o[3];
    DF f[3], r[3], u[3];
    DF k;
    DF inv_spacing;
};

// Double-float arithmetic from the error-free transformations: Knuth's
// TwoSum, Dekker's Fast2Sum (|a| >= |b|), and the product error by FMA.
__device__ __forceinline__ DF df_fast2sum(float a, float b) {
    float s = a + b;
    return DF{s, b - (s - a)};
}
__device__ __forceinline__ DF df_2sum(float a, float b) {
    float s = a + b;
    float bb = s - a;
    return DF{s, (a - (s - bb)) + (b - bb)};
}
__device__ __forceinline__ DF df_2prod(float a, float b) {
    float p = a * b;
    return DF{p, fmaf(a, b, -p)};
}
__device__ __forceinline__ DF df_add(DF x, DF y) {
    DF s = df_2sum(x.hi, y.hi), t = df_2sum(x.lo, y.lo);
    s = df_fast2sum(s.hi, s.lo + t.hi);
    return df_fast2sum(s.hi, s.lo + t.lo);
}
__device__ __forceinline__ DF df_neg(DF x) { return DF{-x.hi, -x.lo}; }
__device__ __forceinline__ DF df_mul(DF x, DF y) {
    DF p = df_2prod(x.hi, y.hi);
    return df_fast2sum(p.hi, fmaf(x.hi, y.lo, fmaf(x.lo, y.hi, p.lo)));
}
__device__ __forceinline__ DF df_mulf(DF x, float b) {
    DF p = df_2prod(x.hi, b);
    return df_fast2sum(p.hi, fmaf(x.lo, b, p.lo));
}
// 1 / y: the FP32 quotient and one Newton step in double-float
__device__ __forceinline__ DF df_rcp(DF y) {
    float r0 = 1.0f / y.hi;
    DF p = df_mulf(y, r0);                 // y r0 = 1 - e
    float e = (1.0f - p.hi) - p.lo;
    return df_fast2sum(r0, r0 * e);
}
// 1 / sqrt(y), y > 0: the FP32 estimate and one Newton step in double-float
__device__ __forceinline__ DF df_rsqrt(DF y) {
    float r0 = rsqrtf(y.hi);
    DF q = df_mulf(df_mulf(y, r0), r0);    // y r0^2 = 1 - e
    float e = (1.0f - q.hi) - q.lo;
    return df_fast2sum(r0, 0.5f * r0 * e);
}
__device__ __forceinline__ bool df_lt(DF a, DF b) { return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo); }
__device__ __forceinline__ DF df_of(double v) {
    float hi = (float)v;
    return DF{hi, (float)(v - (double)hi)};
}

// One rank's brick as the kernels see it.
struct BrickDev {
    const void* data;  // stored nodes, x fastest
    int s_lo[3];       // first stored node (global node index)
    int s_n[3];        // stored nodes per axis (>= 2)
    float r0[3], r1[3];// owned region, node coordinates, clipped to the volume
    int closed[3];     // 1 where r1 is the volume's upper face (closed end)
    int sx, sxy;       // strides of y and z in nodes
    int scale_idx;     // index into the device scale array
    int pad;
    const void* gather;// gather layout or null (GATHER_LINEAR): GATHER_QUAD,
                       // per cell face (x, y) of every z layer the 2x2
                       // corners v(x,y) v(x+1,y) v(x,y+1) v(x+1,y+1) in one
                       // vector (see Quad); GATHER_CELL, per cell its eight
                       // corners in one vector (see Cell)
    int qx, qxy;       // strides of both layouts: s_n[0]-1, (s_n[0]-1)(s_n[1]-1)
    int o_lo[3], o_hi[3];  // owned global nodes [o_lo, o_hi)
    long long gface_off;   // first face of this brick in the face adjoint buffer
    const float2* mm;      // per macro-cell (MACRO^3 cells) min and max of the
                           // decoded node values (empty-space skipping)
    unsigned char* empty;  // per macro-cell: 1 where every sample inside has
                           // TF opacity exactly 0 (rebuilt per render)
    int mx, mxy, mn;       // macro-cell strides and count
};

// Empty-space skipping: macro-cells of 2^MACRO_SHIFT cells per axis.
constexpr int MACRO_SHIFT = 3;
// Deep fragments: fragment layers per work item (DPV_DEEP_MAX).
constexpr int DEEP_LAYERS = 4;

// A work item: one brick seen through one screen tile of one camera.
struct Item {
    int cam;
    int tile;          // tile index within the camera's image
    int brick;
    int pad;
};

struct Counters {
    unsigned long long samples_fwd;
    unsigned long long samples_bwd;
    unsigned long long n_items;
    unsigned int err;
    unsigned int max_frag;
    unsigned long long samples_shadow;
};

// Per-frame constants, passed by value.
struct FrameParams {
    int W, H;          // image size
    int tw, th;        // tile size (tw % 8 == 0, th % 4 == 0)
    int ntx, nty;      // tiles per row / column
    int ncam, tp;      // cameras, pixels per tile
    float dt;          // world step
    float inv_dt;
    float sigma_max;
    float ert;         // local opacity threshold
    int ert_on;
    float vmin;        // TF domain [vmin, vmax]
    float vmax;
    float tf_scale;    // (n - 1) / (vmax - vmin)
    float tf_bias;     // -vmin tf_scale: the TF coordinate is u = fma(s, tf_scale, tf_bias)
    float sdt;         // sigma_max dt: a sample's optical depth is its TF opacity times sdt
    int ntf;           // TF entries
    int dims[3];       // global nodes per axis
    int nbricks;
    int order_stride;  // bytes per pixel of the order image (0 = off)
    int items_cap;     // work items the list and fragment pool hold
    int box_cap;       // floats of shared memory per slab box (staged march)
    int ordered_on;    // visibility-ordered march, global early termination
    int skip_on;       // empty-space skipping in the forward march
    int quad_pair;     // forward quad gather: pair-wide loads (layouts far larger than L2)
    int deep;          // fragment layers per work item: 1, or DEEP_LAYERS (deep fragments)
    int shadow_on;     // volumetric shadows by ray forwarding
    float hl[3];       // shadow step h L, node units
    float shadow_dt;   // h in world units (the shadow samples' opacity step)
    float ambient;     // k_a
    int iso_on;        // iso-surface fragments instead of volume rendering
    float iso;         // their level
    const float4* rays;// per camera and pixel RAY_VECS float4; see k_rays
};

// A work item read back from the list is used only if it names a valid
// camera, tile and brick (the list is rebuilt every frame; an overflowed
// tile leaves its entries unwritten).
__device__ __forceinline__ bool item_ok(const Item& it, const FrameParams& P) {
    return (unsigned)it.cam < (unsigned)P.ncam && (unsigned)it.brick < (unsigned)P.nbricks &&
           (unsigned)it.tile < (unsigned)(P.ntx * P.nty);
}

// ---------------------------------------------------------------------------
// tiles: warps cover 8 x 4 pixel blocks, laid row-major inside the tile, so
// a warp's rays are spatially compact.  The fragment of tile thread t is
// stored at slot t of its item (thread order).
// ---------------------------------------------------------------------------
__device__ __forceinline__ void tile_pixel(int t, int tw, int& lx, int& ly) {
    int w = t >> 5, l = t & 31;
    int wpr = tw >> 3;
    lx = (w % wpr) * 8 + (l & 7);
    ly = (w / wpr) * 4 + (l >> 3);
}

// ---------------------------------------------------------------------------
// rays: pinhole camera, pixel centres, row 0 at the bottom.  The ray setup
// pass (k_rays) computes every pixel's direction once per frame in FP64 and
// stores it rounded to FP32, together with its FP32 reciprocal and the ray's
// interval in the volume.  A ray is the camera's eye in node coordinates
// plus that direction (node units per world unit of t).
// ---------------------------------------------------------------------------
struct Ray {
    float o[3], d[3], inv[3];
    float te, tx;      // interval in the volume box, clipped to t >= 0
};

// Parametric interval of a ray in the node-space box [lo, hi] per axis.  An
// axis the ray is parallel to constrains nothing if the origin lies in
// [lo, hi) (or [lo, hi] where `closed`), else empties the interval.  Every
// face plane's t is (plane - o) * inv computed one way, so boxes that share
// a plane get bit-identical boundaries and their sample ranges tile the ray.
__device__ __forceinline__ void ray_box(const float o[3], const float d[3], const float inv[3], const float lo[3],
                                        const float hi[3], const int closed[3], float& t0, float& t1) {
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (d[a] != 0.0f) {
            float ta = (lo[a] - o[a]) * inv[a];
            float tb = (hi[a] - o[a]) * inv[a];
            t0 = fmaxf(t0, fminf(ta, tb));
            t1 = fminf(t1, fmaxf(ta, tb));
        } else {
            bool in = o[a] >= lo[a] && (closed[a] ? o[a] <= hi[a] : o[a] < hi[a]);
            if (!in) t0 = __int_as_float(0x7f800000);
        }
    }
}

// Interval of the ray in the whole volume [0, dims - 1], clipped to t >= 0.
__device__ __forceinline__ bool volume_interval(const int dims[3], const float o[3], const float d[3],
                                                const float inv[3], float& te, float& tx) {
    const float lo[3] = {0.0f, 0.0f, 0.0f};
    const float hi[3] = {(float)(dims[0] - 1), (float)(dims[1] - 1), (float)(dims[2] - 1)};
    const int closed[3] = {1, 1, 1};
    te = 0.0f;
    tx = __int_as_float(0x7f800000);
    ray_box(o, d, inv, lo, hi, closed, te, tx);
    return te < tx;
}

__device__ __forceinline__ void load_ray(const CamBasis& cam, const FrameParams& P, int c, int px, int py, Ray& r) {
    long long i = ((long long)c * P.H + py) * P.W + px;
    float4 a = __ldg(P.rays + RAY_VECS * i), b = __ldg(P.rays + RAY_VECS * i + 1);
    r.d[0] = a.x;
    r.d[1] = a.y;
    r.d[2] = a.z;
    r.te = a.w;
    r.inv[0] = b.x;
    r.inv[1] = b.y;
    r.inv[2] = b.z;
    r.tx = b.w;
    r.o[0] = cam.o[0];
    r.o[1] = cam.o[1];
    r.o[2] = cam.o[2];
}

// The ray's volume entry point and direction as unevaluated FP32 pairs
// (hi + lo), from the FP64 ray setup: entry point = eye + t_enter d.
struct RayExact {
    float p_hi[3], p_lo[3], d_lo[3];
};

__device__ __forceinline__ void load_ray_exact(const FrameParams& P, int c, int px, int py, RayExact& e) {
    long long i = ((long long)c * P.H + py) * P.W + px;
    float4 u = __ldg(P.rays + RAY_VECS * i + 2), v = __ldg(P.rays + RAY_VECS * i + 3),
           w = __ldg(P.rays + RAY_VECS * i + 4);
    e.p_hi[0] = u.x;
    e.p_hi[1] = u.y;
    e.p_hi[2] = u.z;
    e.p_lo[0] = v.x;
    e.p_lo[1] = v.y;
    e.p_lo[2] = v.z;
    e.d_lo[0] = w.x;
    e.d_lo[1] = w.y;
    e.d_lo[2] = w.z;
}

// Sample index of the first sample at or after t: samples sit at
// t_enter + (j + 1/2) dt.
__device__ __forceinline__ int first_sample_at(float t, float te, const FrameParams& P) {
    return (int)ceilf((t - te) * P.inv_dt - 0.5f);
}

// ---------------------------------------------------------------------------
// stored values
// ---------------------------------------------------------------------------
template <typename T>
struct Storage;

template <>
struct Storage<float> {
    static __device__ __forceinline__ float load(const float* p, int i) { return __ldg(p + i); }
    static constexpr bool unit_scale = true;
};
template <>
struct Storage<__half> {
    static __device__ __forceinline__ float load(const __half* p, int i) {
        return __half2float(__ushort_as_half(__ldg(reinterpret_cast<const unsigned short*>(p) + i)));
    }
    static constexpr bool unit_scale = false;
};
template <>
struct Storage<__nv_bfloat16> {
    static __device__ __forceinline__ float load(const __nv_bfloat16* p, int i) {
        return __bfloat162float(__ushort_as_bfloat16(__ldg(reinterpret_cast<const unsigned short*>(p) + i)));
    }
    static constexpr bool unit_scale = false;
};
template <>
struct Storage<__nv_fp8_e4m3> {
    static __device__ __forceinline__ float load(const __nv_fp8_e4m3* p, int i) {
        unsigned char b = __ldg(reinterpret_cast<const unsigned char*>(p) + i);
        return __half2float(__half(__nv_cvt_fp8_to_halfraw((__nv_fp8_storage_t)b, __NV_E4M3)));
    }
    static constexpr bool unit_scale = false;
};

// Four corners of one (x, y) cell face packed in the gather layout.
template <typename T>
struct Quad;
template <>
struct Quad<float> {
    using W = float4;
    static __device__ __forceinline__ void unpack(W w, float& a, float& b, float& c, float& d) {
        a = w.x;
        b = w.y;
        c = w.z;
        d = w.w;
    }
};
template <>
struct Quad<__half> {
    using W = uint2;
    static __device__ __forceinline__ void unpack(W w, float& a, float& b, float& c, float& d) {
        a = __half2float(__ushort_as_half((unsigned short)(w.x & 0xffffu)));
        b = __half2float(__ushort_as_half((unsigned short)(w.x >> 16)));
        c = __half2float(__ushort_as_half((unsigned short)(w.y & 0xffffu)));
        d = __half2float(__ushort_as_half((unsigned short)(w.y >> 16)));
    }
};
template <>
struct Quad<__nv_bfloat16> {
    using W = uint2;
    static __device__ __forceinline__ void unpack(W w, float& a, float& b, float& c, float& d) {
        a = __uint_as_float(w.x << 16);
        b = __uint_as_float(w.x & 0xffff0000u);
        c = __uint_as_float(w.y << 16);
        d = __uint_as_float(w.y & 0xffff0000u);
    }
};
// Two E4M3 values (low byte first) to FP32 through one paired conversion to
// f16x2: both steps are exact, so the values equal the one-at-a-time decode
// at half the conversions.
__device__ __forceinline__ float2 fp8x2_to_float2(unsigned int pair) {
    const __half2_raw h = __nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)(pair & 0xffffu), __NV_E4M3);
    return __half22float2(__half2(h));
}

template <>
struct Quad<__nv_fp8_e4m3> {
    using W = unsigned int;
    static __device__ __forceinline__ void unpack(W w, float& a, float& b, float& c, float& d) {
        const float2 lo = fp8x2_to_float2(w), hi = fp8x2_to_float2(w >> 16);
        a = lo.x;
        b = lo.y;
        c = hi.x;
        d = hi.y;
    }
};

// Eight corners of one cell, corner c = dx + 2 dy + 4 dz, in one aligned
// vector of the cell gather layout: a single load per sample (256-bit for
// float32).
template <typename T>
struct Cell;
template <>
struct Cell<float> {
    static __device__ __forceinline__ void load(const void* base, long long cell, float v[8]) {
        const float* p = reinterpret_cast<const float*>(base) + 8 * cell;
        asm("ld.global.nc.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
            : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3]), "=f"(v[4]), "=f"(v[5]), "=f"(v[6]), "=f"(v[7])
            : "l"(p));
    }
};
template <>
struct Cell<__half> {
    static __device__ __forceinline__ void load(const void* base, long long cell, float v[8]) {
        const uint4 w = __ldg(reinterpret_cast<const uint4*>(base) + cell);
        const unsigned u[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            v[2 * k] = __half2float(__ushort_as_half((unsigned short)(u[k] & 0xffffu)));
            v[2 * k + 1] = __half2float(__ushort_as_half((unsigned short)(u[k] >> 16)));
        }
    }
};
template <>
struct Cell<__nv_bfloat16> {
    static __device__ __forceinline__ void load(const void* base, long long cell, float v[8]) {
        const uint4 w = __ldg(reinterpret_cast<const uint4*>(base) + cell);
        const unsigned u[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            v[2 * k] = __uint_as_float(u[k] << 16);
            v[2 * k + 1] = __uint_as_float(u[k] & 0xffff0000u);
        }
    }
};
template <>
struct Cell<__nv_fp8_e4m3> {
    static __device__ __forceinline__ void load(const void* base, long long cell, float v[8]) {
        const uint2 w = __ldg(reinterpret_cast<const uint2*>(base) + cell);
        Quad<__nv_fp8_e4m3>::unpack(w.x, v[0], v[1], v[2], v[3]);
        Quad<__nv_fp8_e4m3>::unpack(w.y, v[4], v[5], v[6], v[7]);
    }
};

// Raw cell vectors, fetched one sample ahead and decoded at use.
template <typename T>
struct CellRaw;
template <>
struct CellRaw<float> {
    float v[8];
    __device__ __forceinline__ void fetch(const void* base, long long cell) { Cell<float>::load(base, cell, v); }
    __device__ __forceinline__ void decode(float o[8]) const {
#pragma unroll
        for (int k = 0; k < 8; ++k) o[k] = v[k];
    }
};
template <>
struct CellRaw<__half> {
    uint4 w;
    __device__ __forceinline__ void fetch(const void* base, long long cell) {
        w = __ldg(reinterpret_cast<const uint4*>(base) + cell);
    }
    __device__ __forceinline__ void decode(float v[8]) const {
        const unsigned u[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            v[2 * k] = __half2float(__ushort_as_half((unsigned short)(u[k] & 0xffffu)));
            v[2 * k + 1] = __half2float(__ushort_as_half((unsigned short)(u[k] >> 16)));
        }
    }
};
template <>
struct CellRaw<__nv_bfloat16> {
    uint4 w;
    __device__ __forceinline__ void fetch(const void* base, long long cell) {
        w = __ldg(reinterpret_cast<const uint4*>(base) + cell);
    }
    __device__ __forceinline__ void decode(float v[8]) const {
        const unsigned u[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            v[2 * k] = __uint_as_float(u[k] << 16);
            v[2 * k + 1] = __uint_as_float(u[k] & 0xffff0000u);
        }
    }
};
template <>
struct CellRaw<__nv_fp8_e4m3> {
    uint2 w;
    __device__ __forceinline__ void fetch(const void* base, long long cell) {
        w = __ldg(reinterpret_cast<const uint2*>(base) + cell);
    }
    __device__ __forceinline__ void decode(float v[8]) const {
        Quad<__nv_fp8_e4m3>::unpack(w.x, v[0], v[1], v[2], v[3]);
        Quad<__nv_fp8_e4m3>::unpack(w.y, v[4], v[5], v[6], v[7]);
    }
};

// The quad layout interleaves pairs of z layers: face (x, y, z) is vector
// ((z / 2) qxy + y qx + x) 2 + z % 2, so a cell at even z finds its lower
// and upper faces side by side (one sector, or one load of both); at odd z
// they are its pair's second and the next pair's first face.
// (32-bit arithmetic: a brick holds under 2^31 nodes, so under 2^32 slots.)
__device__ __forceinline__ unsigned quad_slot(const BrickDev& b, int x, int y, int z) {
    return ((unsigned)(z >> 1) * (unsigned)b.qxy + (unsigned)y * (unsigned)b.qx + (unsigned)x) * 2u + (unsigned)(z & 1);
}

// Cell index of the cell layout (under 2^31 cells per brick).
__device__ __forceinline__ unsigned cell_slot(const BrickDev& b, int x, int y, int z) {
    return (unsigned)z * (unsigned)b.qxy + (unsigned)y * (unsigned)b.qx + (unsigned)x;
}

// Both faces of a pair in one load.
template <typename T>
struct QuadPair;
template <>
struct QuadPair<float> {
    static __device__ __forceinline__ void load(const float4* p, float4& lo, float4& hi) {
        asm("ld.global.nc.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
            : "=f"(lo.x), "=f"(lo.y), "=f"(lo.z), "=f"(lo.w), "=f"(hi.x), "=f"(hi.y), "=f"(hi.z), "=f"(hi.w)
            : "l"(p));
    }
};
template <typename H>
struct QuadPair16 {
    static __device__ __forceinline__ void load(const uint2* p, uint2& lo, uint2& hi) {
        const uint4 w = __ldg(reinterpret_cast<const uint4*>(p));
        lo = make_uint2(w.x, w.y);
        hi = make_uint2(w.z, w.w);
    }
};
template <>
struct QuadPair<__half> : QuadPair16<__half> {};
template <>
struct QuadPair<__nv_bfloat16> : QuadPair16<__nv_bfloat16> {};
template <>
struct QuadPair<__nv_fp8_e4m3> {
    static __device__ __forceinline__ void load(const unsigned* p, unsigned& lo, unsigned& hi) {
        const uint2 w = __ldg(reinterpret_cast<const uint2*>(p));
        lo = w.x;
        hi = w.y;
    }
};

// Raw face vectors of one cell in the quad layout (lower face, upper face),
// fetched one sample ahead and decoded at use.  At even z the upper face is
// the next slot of the same pair (the same sector), at odd z the lower face
// of the next pair.  By default two loads for every cell, with no branch on
// the parity of z (lanes of a warp differ in it); with PAIR one pair-wide
// load at even z behind that branch.  Measured: where the layout is served
// from L1/L2 (512^3) the branch-free form is faster (forward bf16 +6 %, f32
// +15 %); where every sample's faces come from DRAM (2048^3 bf16) the
// pair-wide load is (forward 195.6 against 199.0 ms), and the adjoint
// prefers the branch-free form at both sizes (2048^3: 746.7 against 756.8 ms).
template <typename T, bool PAIR = false>
struct QuadRaw {
    typename Quad<T>::W lo, hi;
    __device__ __forceinline__ void fetch(const BrickDev& b, int x, int y, int z) {
        const typename Quad<T>::W* q = reinterpret_cast<const typename Quad<T>::W*>(b.gather) + quad_slot(b, x, y, z);
        if (PAIR && !(z & 1)) {
            QuadPair<T>::load(q, lo, hi);
        } else {
            lo = __ldg(q);
            hi = __ldg(q + ((z & 1) ? (2u * (unsigned)b.qxy - 1u) : 1u));
        }
    }
    __device__ __forceinline__ void decode(float v[8]) const {
        Quad<T>::unpack(lo, v[0], v[1], v[2], v[3]);
        Quad<T>::unpack(hi, v[4], v[5], v[6], v[7]);
    }
};

// The raw gather of the layouts that fetch one sample ahead (PAIR: the
// quad layout's pair-wide load at even z).
template <typename T, int GL, bool PAIR = false>
struct GatherRaw;
template <typename T, bool PAIR>
struct GatherRaw<T, GATHER_CELL, PAIR> {
    CellRaw<T> r;
    __device__ __forceinline__ void fetch(const BrickDev& b, int x, int y, int z) { r.fetch(b.gather, cell_slot(b, x, y, z)); }
    __device__ __forceinline__ void decode(float v[8]) const { r.decode(v); }
};
template <typename T, bool PAIR>
struct GatherRaw<T, GATHER_QUAD, PAIR> {
    QuadRaw<T, PAIR> r;
    __device__ __forceinline__ void fetch(const BrickDev& b, int x, int y, int z) { r.fetch(b, x, y, z); }
    __device__ __forceinline__ void decode(float v[8]) const { r.decode(v); }
};

// The trilinear interpolant of eight decoded corners (the arithmetic of
// trilinear(), in the same order).
template <typename T>
__device__ __forceinline__ float lerp_cell(const float v[8], float fx, float fy, float fz, float scale) {
    float x00 = fmaf(fx, v[1] - v[0], v[0]);
    float x10 = fmaf(fx, v[3] - v[2], v[2]);
    float x01 = fmaf(fx, v[5] - v[4], v[4]);
    float x11 = fmaf(fx, v[7] - v[6], v[6]);
    float y0 = fmaf(fy, x10 - x00, x00);
    float y1 = fmaf(fy, x11 - x01, x01);
    float r = fmaf(fz, y1 - y0, y0);
    return Storage<T>::unit_scale ? r : r * scale;
}

// The eight corners of the last cell a ray sampled, kept in registers:
// consecutive samples (step < 1 voxel) mostly stay in the same cell, and a
// step to the next cell in z shares a face; only what changed is loaded.
// Used by the eight-load (linear) gather; the quad gather loads its two
// faces every sample, which measures faster than the divergent reuse tests.
template <typename T, int G>
struct CornerCache {
    int ix = -1, iy = -1, iz = -1;
    float v[8];

    __device__ __forceinline__ void face(const BrickDev& b, const T* data, int x, int y, int z, float& a, float& c,
                                         float& d, float& e) const {
        if (G == GATHER_QUAD) {
            using W = typename Quad<T>::W;
            const W* q = reinterpret_cast<const W*>(b.gather) + quad_slot(b, x, y, z);
            Quad<T>::unpack(__ldg(q), a, c, d, e);
        } else {
            const T* p = data + (x + y * b.sx + z * b.sxy);
            a = Storage<T>::load(p, 0);
            c = Storage<T>::load(p, 1);
            d = Storage<T>::load(p, b.sx);
            e = Storage<T>::load(p, b.sx + 1);
        }
    }

    __device__ __forceinline__ void fetch(const BrickDev& b, const T* data, int x, int y, int z) {
        if (x == ix && y == iy && z == iz) return;
        if (x == ix && y == iy && z == iz + 1) {
            v[0] = v[4];
            v[1] = v[5];
            v[2] = v[6];
            v[3] = v[7];
        } else if (x == ix && y == iy && z == iz - 1) {
            v[4] = v[0];
            v[5] = v[1];
            v[6] = v[2];
            v[7] = v[3];
            face(b, data, x, y, z, v[0], v[1], v[2], v[3]);
            iz = z;
            return;
        } else {
            face(b, data, x, y, z, v[0], v[1], v[2], v[3]);
        }
        face(b, data, x, y, z + 1, v[4], v[5], v[6], v[7]);
        ix = x;
        iy = y;
        iz = z;
    }
};

// Trilinear value in cell (ix, iy, iz) with weights (fx, fy, fz) (x
// fastest): lerp in x, then y, then z.  The eight corners come from the
// stored nodes through the ray's corner cache (GATHER_LINEAR), from two
// face vectors (GATHER_QUAD) or from one cell vector (GATHER_CELL): the
// same values in every case.  The per-brick scale multiplies the
// interpolated value (equal to scaling each corner, up to rounding).
template <typename T, int G>
__device__ __forceinline__ float trilinear(const BrickDev& b, const T* data, float scale, CornerCache<T, G>& cc,
                                           int ix, int iy, int iz, float fx, float fy, float fz) {
    if (G == GATHER_CELL) {
        Cell<T>::load(b.gather, cell_slot(b, ix, iy, iz), cc.v);
    } else if (G == GATHER_QUAD) {
        // two vector loads: cheaper than the cache's divergent reuse tests
        cc.face(b, data, ix, iy, iz, cc.v[0], cc.v[1], cc.v[2], cc.v[3]);
        cc.face(b, data, ix, iy, iz + 1, cc.v[4], cc.v[5], cc.v[6], cc.v[7]);
    } else {
        cc.fetch(b, data, ix, iy, iz);
    }
    const float* v = cc.v;
    float x00 = fmaf(fx, v[1] - v[0], v[0]);
    float x10 = fmaf(fx, v[3] - v[2], v[2]);
    float x01 = fmaf(fx, v[5] - v[4], v[4]);
    float x11 = fmaf(fx, v[7] - v[6], v[6]);
    float y0 = fmaf(fy, x10 - x00, x00);
    float y1 = fmaf(fy, x11 - x01, x01);
    float r = fmaf(fz, y1 - y0, y0);
    return Storage<T>::unit_scale ? r : r * scale;
}

// ---------------------------------------------------------------------------
// transfer function and emission-absorption
// ---------------------------------------------------------------------------
struct TFSample {
    float4 v;          // interpolated RGBA
    int i0;            // left entry
    float w;           // weight of the right entry
    float duds;        // du/ds (0 where s lies outside [vmin, vmax])
};

__device__ __forceinline__ TFSample tf_lookup(const float4* tab, const FrameParams& P, float s) {
    TFSample r;
    float u = fmaf(s, P.tf_scale, P.tf_bias);
    float hi = (float)(P.ntf - 1);
    // the clamp is decided on s itself, so a rounded u never moves a sample
    // inside the domain onto the clamped side
    r.duds = (s >= P.vmin && s <= P.vmax) ? P.tf_scale : 0.0f;
    u = fminf(fmaxf(u, 0.0f), hi);
    r.i0 = min(__float2int_rd(u), P.ntf - 2);
    r.w = u - (float)r.i0;
    float4 a = tab[r.i0], b = tab[r.i0 + 1];
    r.v.x = fmaf(r.w, b.x - a.x, a.x);
    r.v.y = fmaf(r.w, b.y - a.y, a.y);
    r.v.z = fmaf(r.w, b.z - a.z, a.z);
    r.v.w = fmaf(r.w, b.w - a.w, a.w);
    return r;
}

// The lookup of tf_lookup, with the last interval's entries kept in
// registers: consecutive samples of a ray often fall in the same interval,
// and then no shared-memory load is needed.  SLOPE keeps the left entry and
// the slope b - a instead of both entries, so the subtraction is not
// repeated either (the ordered march's quad form; on the sort-last quad
// march at 4 CTAs per SM it measured 2048^3 bf16 +1.2 %, fp8 +1.8 %, but the
// uncached lookup at 5 CTAs beats both); on the cell layout's 48-register
// march the slope form measured 5 % slower than both entries.  Same
// arithmetic either way.
// The plain lookup with the TFCache interface (no registers kept: the
// pipelined quad march, whose occupancy the kept entries would cost).
struct TFNoCache {
    __device__ __forceinline__ float4 lookup(const float4* tab, const FrameParams& P, float s) {
        return tf_lookup(tab, P, s).v;
    }
};

template <bool SLOPE>
struct TFCache {
    int i = -1;
    float4 a, b;       // entry i and, with SLOPE, b - a; else entry i + 1
    __device__ __forceinline__ float4 lookup(const float4* tab, const FrameParams& P, float s) {
        float u = fmaf(s, P.tf_scale, P.tf_bias);
        u = fminf(fmaxf(u, 0.0f), (float)(P.ntf - 1));
        const int i0 = min(__float2int_rd(u), P.ntf - 2);
        const float w = u - (float)i0;
        if (i0 != i) {
            i = i0;
            a = tab[i0];
            b = tab[i0 + 1];
            if (SLOPE) b = make_float4(b.x - a.x, b.y - a.y, b.z - a.z, b.w - a.w);
        }
        if (SLOPE) return make_float4(fmaf(w, b.x, a.x), fmaf(w, b.y, a.y), fmaf(w, b.z, a.z), fmaf(w, b.w, a.w));
        return make_float4(fmaf(w, b.x - a.x, a.x), fmaf(w, b.y - a.y, a.y), fmaf(w, b.z - a.z, a.z),
                           fmaf(w, b.w - a.w, a.w));
    }
};

// The lookup with the segment's slopes b - a per channel (the adjoint's
// ds term), from the same two entries.
__device__ __forceinline__ TFSample tf_lookup_slope(const float4* tab, const FrameParams& P, float s, float4& d) {
    TFSample r;
    float u = fmaf(s, P.tf_scale, P.tf_bias);
    float hi = (float)(P.ntf - 1);
    r.duds = (s >= P.vmin && s <= P.vmax) ? P.tf_scale : 0.0f;
    u = fminf(fmaxf(u, 0.0f), hi);
    r.i0 = min(__float2int_rd(u), P.ntf - 2);
    r.w = u - (float)r.i0;
    float4 a = tab[r.i0], b = tab[r.i0 + 1];
    d = make_float4(b.x - a.x, b.y - a.y, b.z - a.z, b.w - a.w);
    r.v.x = fmaf(r.w, d.x, a.x);
    r.v.y = fmaf(r.w, d.y, a.y);
    r.v.z = fmaf(r.w, d.z, a.z);
    r.v.w = fmaf(r.w, d.w, a.w);
    return r;
}

// Opacity 1 - exp(-x) of optical depth x.  For |x| < 1/16 (every sample at
// the usual step and sigma_max: x = sigma_max a dt is about 0.008 at 512^3
// and 0.002 at 2048^3) the Taylor series of 1 - exp(-x) to x^5, in Horner
// form: the truncation is below x^6 / 720 (1.4e-9 relative at the edge of
// the range, below one FP32 rounding), at a third of the instructions of
// the library's expm1f, which takes the other samples.
__device__ __forceinline__ float opacity(float x) {
    if (fabsf(x) < 0.0625f) {
        float q = fmaf(-x, 1.0f / 120.0f, 1.0f / 24.0f);
        q = fmaf(-x, q, 1.0f / 6.0f);
        q = fmaf(-x, q, 0.5f);
        q = fmaf(-x, q, 1.0f);
        return x * q;
    }
    return -expm1f(-x);
}

// Opacity of one sample: 1 - exp(-sigma_max * a * dt).
__device__ __forceinline__ float sample_alpha(const FrameParams& P, float a) { return opacity(a * P.sdt); }

// ---------------------------------------------------------------------------
// one ray through one brick
// ---------------------------------------------------------------------------
struct MarchState {
    int j0, j1;        // sample range [j0, j1)
    float te;          // t_enter of the ray in the volume
    float q0[3];       // brick-local node position of sample j0
    float st[3];       // brick-local step per sample
};

// Ray of pixel (px, py) against brick b: its sample range and the local
// frame.  Returns false when the brick holds no sample of the ray.
// The sample range [j0, j1) of ray r in brick b (the range brick_samples
// uses); false when empty.
__device__ __forceinline__ bool segment_range(const FrameParams& P, const Ray& r, const BrickDev& b, int& j0,
                                              int& j1) {
    if (!(r.te < r.tx)) return false;
    float t0 = r.te, t1 = r.tx;
    ray_box(r.o, r.d, r.inv, b.r0, b.r1, b.closed, t0, t1);
    if (!(t0 < t1)) return false;
    j0 = first_sample_at(t0, r.te, P);
    j1 = first_sample_at(t1, r.te, P);
    return j0 < j1;
}

__device__ __forceinline__ bool brick_samples(const FrameParams& P, const CamBasis& cam, int c, const BrickDev& b,
                                              int px, int py, MarchState& m) {
    Ray r;
    load_ray(cam, P, c, px, py, r);
    if (!segment_range(P, r, b, m.j0, m.j1)) return false;
    m.te = r.te;
    // Position of sample j0 in brick-local node coordinates, kept to about
    // one FP32 ulp of the brick-local value: entry point p = p_hi + p_lo,
    // travel s = (j0 + 1/2) dt as an exact product pair, direction
    // d = d_hi + d_lo; q0 = (p_hi - s_lo) + s d + p_lo with the large terms
    // combined by error-free transformations.  p_hi - s_lo is exact (both
    // are below 2^23 ulps of p_hi apart).
    RayExact e;
    load_ray_exact(P, c, px, py, e);
    const float jh = (float)m.j0 + 0.5f;
    const float s_hi = jh * P.dt;
    const float s_lo = fmaf(jh, P.dt, -s_hi);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        float base = e.p_hi[a] - (float)b.s_lo[a];
        float m_hi = s_hi * r.d[a];
        float m_lo = fmaf(s_hi, r.d[a], -m_hi);
        float tail = e.p_lo[a] + (m_lo + fmaf(s_hi, e.d_lo[a], s_lo * r.d[a]));
        // two-sum of base and m_hi, then the tail
        float sum = base + m_hi;
        float bb = sum - base;
        float err = (base - (sum - bb)) + (m_hi - bb);
        m.q0[a] = sum + (err + tail);
        m.st[a] = P.dt * r.d[a];
    }
    return true;
}

// Sample positions of a ray inside a brick: sample k sits at
// fma(k, st, q0) in brick-local node coordinates (q0 from the double-float
// anchor above), cell clamped to the brick, weights relative to the cell.
// (Re-anchoring the position on an integer base cell every few samples was
// measured: 16x finer positions changed no parity figure and cost 4%.)
struct SampleWalker {
    int lim[3];        // last valid cell index per axis (s_n - 2)

    __device__ __forceinline__ void init(const BrickDev& b) {
        lim[0] = b.s_n[0] - 2;
        lim[1] = b.s_n[1] - 2;
        lim[2] = b.s_n[2] - 2;
    }

    // RELU: the clamp to [0, lim] as one max(min(i, lim), 0) call (lim >= 0),
    // the same integers; measured faster in the pipelined forward marches
    // (2048^3 quad: bf16 +1.3 %, fp8 +2.3 %; 512^3 f16 cell +4.7 %) except
    // the float32 cell march, whose 48 registers then spill more (-15 %),
    // and no faster in the adjoint
    template <bool RELU = false>
    __device__ __forceinline__ void at(const MarchState& m, int k, int& ix, int& iy, int& iz, float& fx, float& fy,
                                       float& fz) const {
        const float fk = (float)k;
        float qx = fmaf(fk, m.st[0], m.q0[0]), qy = fmaf(fk, m.st[1], m.q0[1]), qz = fmaf(fk, m.st[2], m.q0[2]);
        if (RELU) {
            ix = __vimin_s32_relu(__float2int_rd(qx), lim[0]);
            iy = __vimin_s32_relu(__float2int_rd(qy), lim[1]);
            iz = __vimin_s32_relu(__float2int_rd(qz), lim[2]);
        } else {
            ix = min(max(__float2int_rd(qx), 0), lim[0]);
            iy = min(max(__float2int_rd(qy), 0), lim[1]);
            iz = min(max(__float2int_rd(qz), 0), lim[2]);
        }
        fx = qx - (float)ix;
        fy = qy - (float)iy;
        fz = qz - (float)iz;
    }
};

// Empty-space skipping: the last sample index (>= k, <= n - 1) whose cell
// still lies in the macro-cell of cell (ix, iy, iz).  Per axis, the sample
// position q(k') = q0 + k' st stays at least MACRO_EPS inside the
// macro-cell's face for every k' <= (face -/+ MACRO_EPS - q0) / st - 1; the
// margin covers the rounding of the division and of q(k') (both well below
// 1e-3 node for bricks under 4096 nodes).  Faces at the brick's ends, where
// the cell index is clamped, are never crossed.
constexpr float MACRO_EPS = 1.0f / 64.0f;

__device__ __forceinline__ int macro_last(const MarchState& m, const SampleWalker& wk, int k, int n, int ix, int iy,
                                          int iz) {
    const int c[3] = {ix >> MACRO_SHIFT, iy >> MACRO_SHIFT, iz >> MACRO_SHIFT};
    float kmax = (float)(n - 1);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float s = m.st[a];
        float face;
        if (s > 0.0f) {
            const int u = (c[a] + 1) << MACRO_SHIFT;
            if (u > wk.lim[a]) continue;
            face = (float)u - MACRO_EPS;
        } else if (s < 0.0f) {
            const int l = c[a] << MACRO_SHIFT;
            if (l == 0) continue;
            face = (float)l + MACRO_EPS;
        } else {
            continue;
        }
        kmax = fminf(kmax, floorf((face - m.q0[a]) / s) - 1.0f);
    }
    return max(k, (int)kmax);
}

// ---------------------------------------------------------------------------
// gradient accumulation runs (adjoint march)
// ---------------------------------------------------------------------------
struct TFRun {
    int i0 = -1;
    float a[8];        // entry i0 (rgba), entry i0+1 (rgba)
};

__device__ __forceinline__ void tf_flush(TFRun& r, double* s_g) {
    if (r.i0 < 0) return;
    double* e = s_g + 4 * r.i0;
#pragma unroll
    for (int c = 0; c < 8; ++c)
        if (r.a[c] != 0.0f) atomicAdd(e + c, (double)r.a[c]);
}

// Adjoint of one cell's eight corners, summed in registers while a ray stays
// in the cell (scalar-atomic path).  a[0..3] are the corners of the cell's
// lower z face in the order (x,y) (x+1,y) (x,y+1) (x+1,y+1); a[4..7] those of
// its upper face.
struct CellRun {
    long long base = -1;   // the cell's (0,0,0) node in the global field
    float a[8];
};

// Scalar form: eight FP32 atomics into the global field (base = node index).
__device__ __forceinline__ void cell_flush(CellRun& r, float* dvol, long long sy, long long sz) {
    if (r.base < 0) return;
    float* v = dvol + r.base;
    atomicAdd(v, r.a[0]);
    atomicAdd(v + 1, r.a[1]);
    atomicAdd(v + sy, r.a[2]);
    atomicAdd(v + sy + 1, r.a[3]);
    atomicAdd(v + sz, r.a[4]);
    atomicAdd(v + sz + 1, r.a[5]);
    atomicAdd(v + sz + sy, r.a[6]);
    atomicAdd(v + sz + sy + 1, r.a[7]);
}


// ---------------------------------------------------------------------------
// helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long warp_sum_u64(unsigned long long v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

}  // namespace dpv
