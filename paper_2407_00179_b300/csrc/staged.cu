// staged.cu -- brick ray-march and its adjoint with the brick staged in
// shared memory, slab by slab.
//
// One CTA marches the rays of one work item (camera, brick, screen tile).
// The brick is cut into slabs of cells along the tile's dominant axis D
// (the axis along which its centre ray moves fastest).  The CTA visits the
// slabs in the rays' order of travel; for each slab it
//   1. finds, for every ray, the samples whose cell lies in the slab (a
//      contiguous index range, since positions are monotone in the sample
//      index) and their extent on the two other axes,
//   2. reduces those extents into one node box and loads it into shared
//      memory with coalesced row loads, decoding and scaling each node once,
//   3. marches every ray's samples of the slab reading the eight corners
//      from shared memory.
// A slab whose box exceeds the shared budget is halved; a one-cell slab that
// still does not fit is marched straight from global memory.  Rays moving
// against the tile's direction along D (only in very wide tiles) are marched
// from global memory.  Per-sample arithmetic is the one of the unstaged
// kernels (dpv_internal.cuh), with each corner decoded and scaled before
// interpolation, so a float32 brick gives bit-identical fragments.
//
// The adjoint stages the same boxes and also privatises the voxel gradient
// in a shared box that is added to the global field once per slab, instead
// of eight global atomics per sample.
#include <limits.h>

#include "dpv_internal.cuh"
#include "launch.h"

namespace dpv {

namespace {

constexpr int SLAB_CELLS = 8;     // cells per slab along D (halved when the box does not fit)

// Component a (a runtime axis index) of a 3-vector, by selects: indexing
// arrays with a runtime value would move them to local memory.
__device__ __forceinline__ float sel3(const float v[3], int a) { return a == 0 ? v[0] : (a == 1 ? v[1] : v[2]); }
__device__ __forceinline__ int sel3(const int v[3], int a) { return a == 0 ? v[0] : (a == 1 ? v[1] : v[2]); }

// clamped cell index of sample k on axis a (the sample walker's position)
__device__ __forceinline__ int cell_at(const MarchState& m, const BrickDev& b, int a, int k) {
    SampleWalker w;
    w.init(b);
    int c[3];
    float f[3];
    w.at(m, k, c[0], c[1], c[2], f[0], f[1], f[2]);
    return sel3(c, a);
}

// First sample index e >= k whose cell on D lies beyond the slab [slo, shi]
// in the direction of travel (or n): the ray's samples [k, e) are the slab's.
__device__ __forceinline__ int slab_end(const MarchState& m, const BrickDev& b, int D, bool up, int slo, int shi,
                                        int k, int n) {
    const int last = sel3(b.s_n, D) - 2;
    if (up ? shi >= last : slo <= 0) return n;
    const float st = sel3(m.st, D), q0 = sel3(m.q0, D);
    float est = up ? ceilf(((float)(shi + 1) - q0) / st) : floorf(((float)slo - q0) / st) + 1.0f;
    int e = (int)fminf(fmaxf(est, (float)k), (float)n);
    while (e > k) {
        int c = cell_at(m, b, D, e - 1);
        if (up ? c <= shi : c >= slo) break;
        --e;
    }
    while (e < n) {
        int c = cell_at(m, b, D, e);
        if (!(up ? c <= shi : c >= slo)) break;
        ++e;
    }
    return e;
}

__device__ __forceinline__ int warp_min(int v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = min(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}
__device__ __forceinline__ int warp_max(int v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Eight corner values (decoded, scaled) of cell `base` in global storage.
template <typename T>
__device__ __forceinline__ void corners_global(const BrickDev& b, const T* data, float scale, int base, float v[8]) {
    const T* p = data + base;
    const int o[8] = {0, 1, b.sx, b.sx + 1, b.sxy, b.sxy + 1, b.sxy + b.sx, b.sxy + b.sx + 1};
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        float x = Storage<T>::load(p, o[c]);
        v[c] = Storage<T>::unit_scale ? x : x * scale;
    }
}

__device__ __forceinline__ float lerp8(const float v[8], float fx, float fy, float fz) {
    float x00 = fmaf(fx, v[1] - v[0], v[0]);
    float x10 = fmaf(fx, v[3] - v[2], v[2]);
    float x01 = fmaf(fx, v[5] - v[4], v[4]);
    float x11 = fmaf(fx, v[7] - v[6], v[6]);
    float y0 = fmaf(fy, x10 - x00, x00);
    float y1 = fmaf(fy, x11 - x01, x01);
    return fmaf(fz, y1 - y0, y0);
}

// Sample position k of a ray: brick cells, weights, and (for the global
// path) the cell's linear index in the brick.
struct SamplePos {
    int ix, iy, iz;
    float fx, fy, fz;
};

__device__ __forceinline__ SamplePos sample_pos(const MarchState& m, const BrickDev& b, SampleWalker& w, int k) {
    SamplePos s;
    w.at(m, k, s.ix, s.iy, s.iz, s.fx, s.fy, s.fz);
    return s;
}

// The staged box of the current slab (brick-local nodes, inclusive).
struct Box {
    int lo[3];
    int nx, nxy;
    int n[3];
};

// Corner values from the shared box; indices outside it (impossible by
// construction) are clamped and reported.
__device__ __forceinline__ void corners_box(const float* s_box, const Box& bx, const SamplePos& p, float v[8],
                                            unsigned* err) {
    int rx = p.ix - bx.lo[0], ry = p.iy - bx.lo[1], rz = p.iz - bx.lo[2];
    if ((unsigned)rx > (unsigned)(bx.n[0] - 2) || (unsigned)ry > (unsigned)(bx.n[1] - 2) ||
        (unsigned)rz > (unsigned)(bx.n[2] - 2)) {
        atomicOr(err, ERR_STAGE_OUTSIDE);
        rx = min(max(rx, 0), bx.n[0] - 2);
        ry = min(max(ry, 0), bx.n[1] - 2);
        rz = min(max(rz, 0), bx.n[2] - 2);
    }
    const float* q = s_box + rx + ry * bx.nx + rz * bx.nxy;
    v[0] = q[0];
    v[1] = q[1];
    v[2] = q[bx.nx];
    v[3] = q[bx.nx + 1];
    v[4] = q[bx.nxy];
    v[5] = q[bx.nxy + 1];
    v[6] = q[bx.nxy + bx.nx];
    v[7] = q[bx.nxy + bx.nx + 1];
}

// Load box nodes into shared memory, one row (fixed y, z) per warp step,
// lanes along x.
template <typename T>
__device__ __forceinline__ void load_box(const BrickDev& b, const T* data, float scale, const Box& bx, float* s_box,
                                         float* s_gbox) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int rows = bx.n[1] * bx.n[2];
    for (int r = warp; r < rows; r += nw) {
        int y = r % bx.n[1], z = r / bx.n[1];
        const T* src = data + (bx.lo[2] + z) * b.sxy + (bx.lo[1] + y) * b.sx + bx.lo[0];
        float* dst = s_box + r * bx.nx;
        for (int x = lane; x < bx.nx; x += 32) {
            float v = Storage<T>::load(src, x);
            dst[x] = Storage<T>::unit_scale ? v : v * scale;
            if (s_gbox) s_gbox[r * bx.nx + x] = 0.0f;
        }
    }
}

// Dominant axis and direction of the tile's centre ray.
__device__ __forceinline__ void tile_axis(const FrameParams& P, const CamBasis& cam, const Item& it, int& D, bool& up) {
    int tx0 = (it.tile % P.ntx) * P.tw, ty0 = (it.tile / P.ntx) * P.th;
    Ray rc;
    load_ray(cam, P, it.cam, min(tx0 + P.tw / 2, P.W - 1), min(ty0 + P.th / 2, P.H - 1), rc);
    float ax = fabsf(rc.d[0]), ay = fabsf(rc.d[1]), az = fabsf(rc.d[2]);
    D = ax >= ay ? (ax >= az ? 0 : 2) : (ay >= az ? 1 : 2);
    up = sel3(rc.d, D) > 0.0f;
}

// CTA-wide min/max of four ints through shared slots red[0..3]
// (red[0]=min, red[1]=max, red[2]=min, red[3]=max).  All threads call it.
__device__ __forceinline__ void cta_minmax4(int* red, int a0, int a1, int a2, int a3) {
    __syncthreads();
    if (threadIdx.x == 0) {
        red[0] = INT_MAX;
        red[1] = INT_MIN;
        red[2] = INT_MAX;
        red[3] = INT_MIN;
    }
    __syncthreads();
    a0 = warp_min(a0);
    a1 = warp_max(a1);
    a2 = warp_min(a2);
    a3 = warp_max(a3);
    if ((threadIdx.x & 31) == 0) {
        atomicMin(red + 0, a0);
        atomicMax(red + 1, a1);
        atomicMin(red + 2, a2);
        atomicMax(red + 3, a3);
    }
    __syncthreads();
}

// Plan the next slab starting at cell `cur` along D: the largest slab (at
// most SLAB_CELLS cells, halving) whose box fits `cap` floats.  Returns the
// slab's cell range and box; fits = false when even one cell is too large;
// empty = true when no ray has samples in it.  Every thread's end index e is
// returned for its own ray.
__device__ __forceinline__ void plan_slab(const MarchState& m, const BrickDev& b, bool active, int k, int n, int D,
                                          int A1, int A2, bool up, int cur, int DLO, int DHI, int cap, int* red,
                                          int& slo, int& shi, int& e, Box& bx, bool& fits, bool& empty) {
    int S = SLAB_CELLS;
    for (;;) {
        slo = up ? cur : max(cur - S + 1, DLO);
        shi = up ? min(cur + S - 1, DHI) : cur;
        e = k;
        int l1 = INT_MAX, h1 = INT_MIN, l2 = INT_MAX, h2 = INT_MIN;
        if (active) {
            e = slab_end(m, b, D, up, slo, shi, k, n);
            if (e > k) {
                int a = cell_at(m, b, A1, k), c = cell_at(m, b, A1, e - 1);
                l1 = min(a, c);
                h1 = max(a, c);
                a = cell_at(m, b, A2, k);
                c = cell_at(m, b, A2, e - 1);
                l2 = min(a, c);
                h2 = max(a, c);
            }
        }
        cta_minmax4(red, l1, h1, l2, h2);
        int L1 = red[0], H1 = red[1], L2 = red[2], H2 = red[3];
        empty = L1 > H1;
        if (empty) {
            fits = true;
            return;
        }
        int nD = shi - slo + 2, n1 = H1 - L1 + 2, n2 = H2 - L2 + 2;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            bx.lo[a] = a == D ? slo : (a == A1 ? L1 : L2);
            bx.n[a] = a == D ? nD : (a == A1 ? n1 : n2);
        }
        bx.nx = bx.n[0];
        bx.nxy = bx.n[0] * bx.n[1];
        if (nD * n1 * n2 <= cap) {
            fits = true;
            return;
        }
        if (S == 1) {
            fits = false;
            return;
        }
        S = (S + 1) / 2;
    }
}

}  // namespace

// ===========================================================================
// forward
// ===========================================================================

template <typename T>
__global__ void __launch_bounds__(256) k_march_fwd_staged(FrameParams P, const CamBasis* cams,
                                                          const BrickDev* bricks, const float* scales,
                                                          const Item* items, const float4* tf, float4* frag_rgba,
                                                          int* frag_key, Counters* counters) {
    extern __shared__ float4 s_dyn[];
    float4* s_tf = s_dyn;
    float* s_box = (float*)(s_dyn + P.ntf);
    __shared__ int s_red[4];
    const Item it = items[blockIdx.x];
    if (!item_ok(it, P)) return;                 // uniform over the CTA
    for (int i = threadIdx.x; i < P.ntf; i += blockDim.x) s_tf[i] = tf[i];

    const BrickDev b = bricks[it.brick];
    const CamBasis cam = cams[it.cam];
    const float scale = scales[b.scale_idx];
    const T* data = (const T*)b.data;
    int lx, ly;
    tile_pixel(threadIdx.x, P.tw, lx, ly);
    const int px = (it.tile % P.ntx) * P.tw + lx, py = (it.tile / P.ntx) * P.th + ly;
    const long long slot = (long long)blockIdx.x * P.tp + threadIdx.x;
    const bool inimg = px < P.W && py < P.H;

    MarchState m;
    int n = 0;
    if (inimg && brick_samples(P, cam, it.cam, b, px, py, m)) n = m.j1 - m.j0;
    SampleWalker wk;
    wk.init(b);
    int D, A1, A2;
    bool up;
    tile_axis(P, cam, it, D, up);
    A1 = D == 0 ? 1 : 0;
    A2 = D == 2 ? 1 : 2;
    const bool staged = n > 0 && (up ? sel3(m.st, D) > 0.0f : sel3(m.st, D) < 0.0f);

    float C0 = 0.f, C1 = 0.f, C2 = 0.f, Tr = 1.0f;
    int k = 0;
    bool done = n == 0;
    unsigned long long nsamp = 0;

    auto step = [&](const float v[8], const SamplePos& p) {
        float s = lerp8(v, p.fx, p.fy, p.fz);
        TFSample c = tf_lookup(s_tf, P, s);
        float al = sample_alpha(P, c.v.w);
        float ta = Tr * al;
        C0 = fmaf(ta, c.v.x, C0);
        C1 = fmaf(ta, c.v.y, C1);
        C2 = fmaf(ta, c.v.z, C2);
        Tr = Tr - ta;
        ++nsamp;
        return P.ert_on && 1.0f - Tr > P.ert;
    };
    __syncthreads();                              // TF staged

    // rays travelling against the tile's direction: straight from global memory
    if (n > 0 && !staged) {
        for (; k < n; ++k) {
            SamplePos p = sample_pos(m, b, wk, k);
            float v[8];
            corners_global<T>(b, data, scale, p.ix + p.iy * b.sx + p.iz * b.sxy, v);
            if (step(v, p)) break;
        }
        done = true;
    }

    // cell range along D over the CTA's staged rays
    {
        int dl = INT_MAX, dh = INT_MIN;
        if (staged) {
            int c0 = cell_at(m, b, D, 0), c1 = cell_at(m, b, D, n - 1);
            dl = min(c0, c1);
            dh = max(c0, c1);
        }
        cta_minmax4(s_red, dl, dh, INT_MAX, INT_MIN);
    }
    const int DLO = s_red[0], DHI = s_red[1];
    int cur = up ? DLO : DHI;
    while (DLO <= DHI && (up ? cur <= DHI : cur >= DLO)) {
        const bool active = staged && !done && k < n;
        int slo, shi, e;
        Box bx;
        bool fits, empty;
        plan_slab(m, b, active, k, n, D, A1, A2, up, cur, DLO, DHI, P.box_cap, s_red, slo, shi, e, bx, fits, empty);
        if (!empty) {
            if (fits) {
                load_box<T>(b, data, scale, bx, s_box, nullptr);
                __syncthreads();
                for (; active && k < e; ++k) {
                    SamplePos p = sample_pos(m, b, wk, k);
                    float v[8];
                    corners_box(s_box, bx, p, v, &counters->err);
                    if (step(v, p)) {
                        done = true;
                        ++k;
                        break;
                    }
                }
            } else {
                for (; active && k < e; ++k) {
                    SamplePos p = sample_pos(m, b, wk, k);
                    float v[8];
                    corners_global<T>(b, data, scale, p.ix + p.iy * b.sx + p.iz * b.sxy, v);
                    if (step(v, p)) {
                        done = true;
                        ++k;
                        break;
                    }
                }
            }
        }
        cur = up ? shi + 1 : slo - 1;
        // leave when every staged ray has finished (all terminated early)
        if (!__syncthreads_or(staged && !done && k < n)) break;
    }
    if (staged && !done && k != n) atomicOr(&counters->err, ERR_STAGE_INCOMPLETE);

    if (inimg) {
        if (n > 0) {
            frag_rgba[slot] = make_float4(C0, C1, C2, 1.0f - Tr);
            frag_key[slot] = m.j0;
        } else {
            frag_key[slot] = KEY_EMPTY;
        }
    }
    nsamp = warp_sum_u64(nsamp);
    if ((threadIdx.x & 31) == 0 && nsamp) atomicAdd(&counters->samples_fwd, nsamp);
}

// ===========================================================================
// adjoint
// ===========================================================================

template <typename T>
__global__ void __launch_bounds__(256) k_march_bwd_staged(FrameParams P, const CamBasis* cams,
                                                          const BrickDev* bricks, const float* scales,
                                                          const Item* items, const float4* tf,
                                                          const float4* frag_rgba, const int* frag_key,
                                                          const float4* frag_grad, double* dtf, float* dvol,
                                                          Counters* counters) {
    extern __shared__ float4 s_dyn[];
    float4* s_tf = s_dyn;
    double* s_g = (double*)(s_dyn + P.ntf);
    float* s_box = (float*)(s_g + 4 * P.ntf);
    float* s_gbox = s_box + P.box_cap;
    __shared__ int s_red[4];
    const Item it = items[blockIdx.x];
    if (!item_ok(it, P)) return;                 // uniform over the CTA
    for (int i = threadIdx.x; i < P.ntf; i += blockDim.x) s_tf[i] = tf[i];
    for (int i = threadIdx.x; i < 4 * P.ntf; i += blockDim.x) s_g[i] = 0.0;

    const BrickDev b = bricks[it.brick];
    const CamBasis cam = cams[it.cam];
    const float scale = scales[b.scale_idx];
    const T* data = (const T*)b.data;
    int lx, ly;
    tile_pixel(threadIdx.x, P.tw, lx, ly);
    const int px = (it.tile % P.ntx) * P.tw + lx, py = (it.tile / P.ntx) * P.th + ly;
    const long long slot = (long long)blockIdx.x * P.tp + threadIdx.x;
    const long long sy = P.dims[0], sz = (long long)P.dims[0] * P.dims[1];
    const long long gofs = (long long)b.s_lo[2] * sz + (long long)b.s_lo[1] * sy + b.s_lo[0];

    MarchState m;
    int n = 0;
    float4 F = make_float4(0.f, 0.f, 0.f, 0.f), G = F;
    SampleWalker wk;
    wk.init(b);
    if (px < P.W && py < P.H && frag_key[slot] != KEY_EMPTY) {
        G = frag_grad[slot];
        if ((G.x != 0.f || G.y != 0.f || G.z != 0.f || G.w != 0.f) && brick_samples(P, cam, it.cam, b, px, py, m)) {
            n = m.j1 - m.j0;
            F = frag_rgba[slot];
        }
    }
    int D, A1, A2;
    bool up;
    tile_axis(P, cam, it, D, up);
    A1 = D == 0 ? 1 : 0;
    A2 = D == 2 ? 1 : 2;
    const bool staged = n > 0 && (up ? sel3(m.st, D) > 0.0f : sel3(m.st, D) < 0.0f);

    float C0 = 0.f, C1 = 0.f, C2 = 0.f, Tr = 1.0f;
    const float Tend = 1.0f - F.w;
    const float gscale = Storage<T>::unit_scale ? 1.0f : scale;
    int k = 0;
    bool done = n == 0;
    unsigned long long nsamp = 0;
    TFRun tr;
    CellRun cr;

    // One replayed sample: forward recurrence plus its adjoint.  The voxel
    // gradient gs * weights goes to the shared gradient box (box != nullptr)
    // or, through a register run, to the global field.
    auto step = [&](const float v[8], const SamplePos& p, const Box* bx) {
        float s = lerp8(v, p.fx, p.fy, p.fz);
        TFSample c = tf_lookup(s_tf, P, s);
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
                    G.w * Tend;
        float g_r = G.x * ta, g_g = G.y * ta, g_b = G.z * ta;
        float g_a = gal * P.sdt;
        if (c.i0 != tr.i0) {
            tf_flush(tr, s_g);
            tr.i0 = c.i0;
#pragma unroll
            for (int q = 0; q < 8; ++q) tr.a[q] = 0.0f;
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
        if (dvol && c.duds != 0.0f) {
            float4 ta0 = s_tf[c.i0], ta1 = s_tf[c.i0 + 1];
            float gs = (g_r * (ta1.x - ta0.x) + g_g * (ta1.y - ta0.y) + g_b * (ta1.z - ta0.z) +
                        g_a * (ta1.w - ta0.w)) * c.duds * gscale;
            if (gs != 0.0f) {
                float ax = 1.0f - p.fx, ay = 1.0f - p.fy, az = 1.0f - p.fz;
                float g00 = gs * ay * az, g10 = gs * p.fy * az, g01 = gs * ay * p.fz, g11 = gs * p.fy * p.fz;
                if (bx) {
                    int rx = min(max(p.ix - bx->lo[0], 0), bx->n[0] - 2);
                    int ry = min(max(p.iy - bx->lo[1], 0), bx->n[1] - 2);
                    int rz = min(max(p.iz - bx->lo[2], 0), bx->n[2] - 2);
                    float* q = s_gbox + rx + ry * bx->nx + rz * bx->nxy;
                    atomicAdd(q, g00 * ax);
                    atomicAdd(q + 1, g00 * p.fx);
                    atomicAdd(q + bx->nx, g10 * ax);
                    atomicAdd(q + bx->nx + 1, g10 * p.fx);
                    atomicAdd(q + bx->nxy, g01 * ax);
                    atomicAdd(q + bx->nxy + 1, g01 * p.fx);
                    atomicAdd(q + bx->nxy + bx->nx, g11 * ax);
                    atomicAdd(q + bx->nxy + bx->nx + 1, g11 * p.fx);
                } else {
                    long long gb = gofs + (long long)p.iz * sz + (long long)p.iy * sy + p.ix;
                    if (gb != cr.base) {
                        cell_flush(cr, dvol, sy, sz);
                        cr.base = gb;
#pragma unroll
                        for (int q = 0; q < 8; ++q) cr.a[q] = 0.0f;
                    }
                    cr.a[0] = fmaf(g00, ax, cr.a[0]);
                    cr.a[1] = fmaf(g00, p.fx, cr.a[1]);
                    cr.a[2] = fmaf(g10, ax, cr.a[2]);
                    cr.a[3] = fmaf(g10, p.fx, cr.a[3]);
                    cr.a[4] = fmaf(g01, ax, cr.a[4]);
                    cr.a[5] = fmaf(g01, p.fx, cr.a[5]);
                    cr.a[6] = fmaf(g11, ax, cr.a[6]);
                    cr.a[7] = fmaf(g11, p.fx, cr.a[7]);
                }
            }
        }
        C0 = n0;
        C1 = n1;
        C2 = n2;
        Tr = Tr - ta;
        ++nsamp;
        return P.ert_on && 1.0f - Tr > P.ert;
    };
    __syncthreads();                              // TF and its gradient table ready

    if (n > 0 && !staged) {
        for (; k < n; ++k) {
            SamplePos p = sample_pos(m, b, wk, k);
            float v[8];
            corners_global<T>(b, data, scale, p.ix + p.iy * b.sx + p.iz * b.sxy, v);
            if (step(v, p, nullptr)) break;
        }
        done = true;
    }

    {
        int dl = INT_MAX, dh = INT_MIN;
        if (staged) {
            int c0 = cell_at(m, b, D, 0), c1 = cell_at(m, b, D, n - 1);
            dl = min(c0, c1);
            dh = max(c0, c1);
        }
        cta_minmax4(s_red, dl, dh, INT_MAX, INT_MIN);
    }
    const int DLO = s_red[0], DHI = s_red[1];
    int cur = up ? DLO : DHI;
    while (DLO <= DHI && (up ? cur <= DHI : cur >= DLO)) {
        const bool active = staged && !done && k < n;
        int slo, shi, e;
        Box bx;
        bool fits, empty;
        plan_slab(m, b, active, k, n, D, A1, A2, up, cur, DLO, DHI, P.box_cap, s_red, slo, shi, e, bx, fits, empty);
        if (!empty) {
            if (fits) {
                load_box<T>(b, data, scale, bx, s_box, dvol ? s_gbox : nullptr);
                __syncthreads();
                for (; active && k < e; ++k) {
                    SamplePos p = sample_pos(m, b, wk, k);
                    float v[8];
                    corners_box(s_box, bx, p, v, &counters->err);
                    if (step(v, p, &bx)) {
                        done = true;
                        ++k;
                        break;
                    }
                }
                __syncthreads();
                if (dvol) {
                    // add the slab's voxel gradients to the global field
                    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
                    const int rows = bx.n[1] * bx.n[2];
                    for (int r = warp; r < rows; r += nw) {
                        int y = r % bx.n[1], z = r / bx.n[1];
                        float* dst = dvol + gofs + (long long)(bx.lo[2] + z) * sz + (long long)(bx.lo[1] + y) * sy +
                                     bx.lo[0];
                        const float* src = s_gbox + r * bx.nx;
                        for (int x = lane; x < bx.nx; x += 32) {
                            float g = src[x];
                            if (g != 0.0f) atomicAdd(dst + x, g);
                        }
                    }
                }
            } else {
                for (; active && k < e; ++k) {
                    SamplePos p = sample_pos(m, b, wk, k);
                    float v[8];
                    corners_global<T>(b, data, scale, p.ix + p.iy * b.sx + p.iz * b.sxy, v);
                    if (step(v, p, nullptr)) {
                        done = true;
                        ++k;
                        break;
                    }
                }
            }
        }
        cur = up ? shi + 1 : slo - 1;
        if (!__syncthreads_or(staged && !done && k < n)) break;
    }
    if (staged && !done && k != n) atomicOr(&counters->err, ERR_STAGE_INCOMPLETE);
    tf_flush(tr, s_g);
    if (dvol) cell_flush(cr, dvol, sy, sz);

    nsamp = warp_sum_u64(nsamp);
    if ((threadIdx.x & 31) == 0 && nsamp) atomicAdd(&counters->samples_bwd, nsamp);
    __syncthreads();
    for (int i = threadIdx.x; i < 4 * P.ntf; i += blockDim.x) {
        double v = s_g[i];
        if (v != 0.0) atomicAdd(dtf + i, v);
    }
}

// ===========================================================================
// launchers
// ===========================================================================

size_t staged_fwd_smem(const FrameParams& P) { return sizeof(float4) * P.ntf + sizeof(float) * P.box_cap; }
size_t staged_bwd_smem(const FrameParams& P) {
    return sizeof(float4) * P.ntf + sizeof(double) * 4 * P.ntf + 2 * sizeof(float) * P.box_cap;
}

template <typename T>
static cudaError_t fwd_one(const FrameParams& P, const CamBasis* cams, const BrickDev* bricks, const float* scales,
                           const Item* items, int n_items, const float4* tf, float4* frag_rgba, int* frag_key,
                           Counters* counters, cudaStream_t st) {
    size_t smem = staged_fwd_smem(P);
    if (smem > 48 * 1024) cudaFuncSetAttribute(k_march_fwd_staged<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_march_fwd_staged<T><<<n_items, P.tp, smem, st>>>(P, cams, bricks, scales, items, tf, frag_rgba, frag_key,
                                                       counters);
    return cudaGetLastError();
}

template <typename T>
static cudaError_t bwd_one(const FrameParams& P, const CamBasis* cams, const BrickDev* bricks, const float* scales,
                           const Item* items, int n_items, const float4* tf, const float4* frag_rgba,
                           const int* frag_key, const float4* frag_grad, double* dtf, float* dvol, Counters* counters,
                           cudaStream_t st) {
    size_t smem = staged_bwd_smem(P);
    if (smem > 48 * 1024) cudaFuncSetAttribute(k_march_bwd_staged<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_march_bwd_staged<T><<<n_items, P.tp, smem, st>>>(P, cams, bricks, scales, items, tf, frag_rgba, frag_key,
                                                       frag_grad, dtf, dvol, counters);
    return cudaGetLastError();
}

cudaError_t launch_march_fwd_staged(int dtype, const FrameParams& P, const CamBasis* cams, const BrickDev* bricks,
                                    const float* scales, const Item* items, int n_items, const float4* tf,
                                    float4* frag_rgba, int* frag_key, Counters* counters, cudaStream_t st) {
    if (n_items == 0) return cudaSuccess;
    switch (dtype) {
        case 0: return fwd_one<float>(P, cams, bricks, scales, items, n_items, tf, frag_rgba, frag_key, counters, st);
        case 1: return fwd_one<__half>(P, cams, bricks, scales, items, n_items, tf, frag_rgba, frag_key, counters, st);
        case 2: return fwd_one<__nv_bfloat16>(P, cams, bricks, scales, items, n_items, tf, frag_rgba, frag_key, counters, st);
        default: return fwd_one<__nv_fp8_e4m3>(P, cams, bricks, scales, items, n_items, tf, frag_rgba, frag_key, counters, st);
    }
}

cudaError_t launch_march_bwd_staged(int dtype, const FrameParams& P, const CamBasis* cams, const BrickDev* bricks,
                                    const float* scales, const Item* items, int n_items, const float4* tf,
                                    const float4* frag_rgba, const int* frag_key, const float4* frag_grad,
                                    double* dtf, float* dvol, Counters* counters, cudaStream_t st) {
    if (n_items == 0) return cudaSuccess;
    switch (dtype) {
        case 0: return bwd_one<float>(P, cams, bricks, scales, items, n_items, tf, frag_rgba, frag_key, frag_grad, dtf, dvol, counters, st);
        case 1: return bwd_one<__half>(P, cams, bricks, scales, items, n_items, tf, frag_rgba, frag_key, frag_grad, dtf, dvol, counters, st);
        case 2: return bwd_one<__nv_bfloat16>(P, cams, bricks, scales, items, n_items, tf, frag_rgba, frag_key, frag_grad, dtf, dvol, counters, st);
        default: return bwd_one<__nv_fp8_e4m3>(P, cams, bricks, scales, items, n_items, tf, frag_rgba, frag_key, frag_grad, dtf, dvol, counters, st);
    }
}

}  // namespace dpv
