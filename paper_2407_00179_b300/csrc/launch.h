// launch.h -- host-side launchers of the kernels in kernels.cu, used by the
// C-ABI implementation in device.cu.
#pragma once

#include <cuda_runtime.h>

#include "../../include/dpv.h"
#include "dpv_internal.cuh"

namespace dpv {

// Raw camera as given by the caller (mirrors dpv_camera).
struct CamIn {
    float eye[3], center[3], up[3];
    float fovy_deg;
};

// Source box of a brick commit: `src` (device) holds nodes [d_lo, d_lo + d_n)
// x fastest; the brick stores nodes [s_lo, s_lo + s_n).
struct CommitArgs {
    const void* src;
    int d_lo[3], d_n[3];
    int s_lo[3], s_n[3];
};

// Persistent launches: the order in which CTAs pull work items.
// A group of consecutive bricks [k0, k1) whose face adjoint slots sit in the
// buffer from slot `base` (the first slot of brick k0) on: the adjoint
// replays only the group's items, and the gather adds the group's slots.
struct FaceGroup {
    int k0, k1;
    long long base;
    int runs;                // 1: the adjoint sums a cell run in registers before its reductions
};

struct Schedule {
    const int* sched;        // pull index -> work item
    unsigned int* work;      // pull counter (reset by the launcher)
    int ctas_per_sm;         // 0: as many as fit
};

// Build a pull order over the work list: order 0 = list order, 1 =
// brick-major (all cameras' tiles of one brick together).  hist and cursor
// hold nbricks + 1 ints; tmp one unsigned long long.
cudaError_t launch_schedule(const FrameParams& P, const Item* items, int n_items, int order, int* hist,
                            int* offsets, int* cursor, unsigned long long* tmp, int* sched, cudaStream_t st);

// Message returned by dpvGetLastError() on this host thread.
void set_last_error(const char* msg);

// Why a camera cannot be used (eye == center, up parallel to the view
// direction, fovy outside (0, 180)), or nullptr if it can.
const char* camera_problem(const dpv_camera& c);

cudaError_t launch_commit(const CommitArgs& a, int storage, int src_is_f32, float given_scale, unsigned int* d_tmp,
                          float* d_scale, void* dst, cudaStream_t st);

cudaError_t launch_cull(const FrameParams& P, const CamIn* d_cam_in, float3 origin, float spacing,
                        CamBasis* d_cams, CamBasisDF* d_camd, float4* d_rays, const BrickDev* d_bricks,
                        int4* d_rects, int* d_tile_count, int* d_tile_first, Item* d_items, int cap,
                        Counters* d_counters, bool fill, cudaStream_t st);

cudaError_t launch_march_fwd(int dtype, int gather, const FrameParams& P, const CamBasis* cams,
                             const BrickDev* bricks, const float* scales, const Item* items, int n_items,
                             const float4* tf, float4* frag_rgba, int* frag_key, Counters* counters,
                             cudaStream_t st, const Schedule* sch = nullptr);

// Visibility-ordered march with global early termination (DPV_FRAME_ORDERED):
// one launch over (camera, tile), writing the frame.
cudaError_t launch_march_ordered(int dtype, int gather, const FrameParams& P, const CamBasis* cams,
                                 const BrickDev* bricks, const float* scales, const int* tile_first,
                                 const int* tile_count, const Item* items, const float4* tf, float4* out_rgba,
                                 float* out_depth, unsigned char* order, Counters* counters, unsigned int* work,
                                 cudaStream_t st);

// Empty-space skipping (DPV_FRAME_SKIP): macro-cells a brick needs, their
// value ranges (built per committed brick), and the per-render transparency
// from the TF (z: ntf ints of scratch).
size_t macro_cells(const int s_n[3]);
cudaError_t launch_build_minmax(int dtype, const void* data, const int s_n[3], float2* mm, cudaStream_t st);
cudaError_t launch_classify_empty(int dtype, const FrameParams& P, const BrickDev* bricks, int nbricks,
                                  const float* scales, int max_macro, const float4* tf, int* z, cudaStream_t st);

// Volumetric shadows by ray forwarding (shadow.cu): per slot of the
// brick-major order its sample count and the exclusive 64-bit offsets of
// its records (chunk_sums: shadow_chunk_count entries; total: one), then
// spawn, the K forwarding rounds and the shading march into the fragments.
size_t shadow_chunk_count(const FrameParams& P, int n_items);
cudaError_t launch_shadow_offsets(const FrameParams& P, const CamBasis* cams, const BrickDev* bricks,
                                  const Item* items, int n_items, const int* sched, int* counts, long long* offsets,
                                  long long* chunk_sums, long long* total, cudaStream_t st);
cudaError_t launch_shadow_render(int dtype, int gather, const FrameParams& P, const CamBasis* cams,
                                 const BrickDev* bricks, const float* scales, const Item* items, int n_items,
                                 const int* sched, const int* item_first, const long long* offsets,
                                 const long long* total, long long* rec_first, long long n_recs, float4* recs,
                                 const float4* tf, float4* frag_rgba, int* frag_key, Counters* counters,
                                 cudaStream_t st);

// Iso-surface fragments (DPV_FRAME_ISO) and their depth composite.
cudaError_t launch_iso_fwd(int dtype, int gather, const FrameParams& P, const CamBasis* cams,
                           const BrickDev* bricks, const float* scales, const Item* items, int n_items,
                           const float4* tf, float4* frag_rgba, int* frag_key, Counters* counters, cudaStream_t st);
cudaError_t launch_composite_iso(const FrameParams& P, const CamBasis* cams, const int* tile_first,
                                 const int* tile_count, const Item* items, const float4* frag_rgba,
                                 const int* frag_key, float4* out_rgba, float* out_depth, unsigned char* order,
                                 cudaStream_t st);

// Shared-memory staged ray-march and adjoint (staged.cu).
cudaError_t launch_march_fwd_staged(int dtype, const FrameParams& P, const CamBasis* cams, const BrickDev* bricks,
                                    const float* scales, const Item* items, int n_items, const float4* tf,
                                    float4* frag_rgba, int* frag_key, Counters* counters, cudaStream_t st);
cudaError_t launch_march_bwd_staged(int dtype, const FrameParams& P, const CamBasis* cams, const BrickDev* bricks,
                                    const float* scales, const Item* items, int n_items, const float4* tf,
                                    const float4* frag_rgba, const int* frag_key, const float4* frag_grad,
                                    double* dtf, float* dvol, Counters* counters, cudaStream_t st);
size_t staged_fwd_smem(const FrameParams& P);
size_t staged_bwd_smem(const FrameParams& P);

cudaError_t launch_composite_fwd(const FrameParams& P, float inv_spacing, const CamBasis* cams,
                                 const int* tile_first, const int* tile_count, const Item* items,
                                 const float4* frag_rgba, const int* frag_key, float4* out_rgba, float* out_depth,
                                 unsigned char* order, cudaStream_t st);

cudaError_t launch_composite_bwd(const FrameParams& P, const int* tile_first, const int* tile_count,
                                 const float4* frag_rgba, const int* frag_key, const float4* grad_img,
                                 float4* frag_grad, cudaStream_t st);

cudaError_t launch_march_bwd(int dtype, int gather, const FrameParams& P, const CamBasis* cams,
                             const BrickDev* bricks, const float* scales, const Item* items, int n_items,
                             const float4* tf, const float4* frag_rgba, const int* frag_key,
                             const float4* frag_grad, double* dtf, float* dvol, float4* gface,
                             Counters* counters, cudaStream_t st, const Schedule* sch = nullptr,
                             const FaceGroup* fg = nullptr);

// Face adjoint buffer (kernels.cu): float4 slots it needs for a brick (one
// per cell face, as the gather layout), and the pass that turns the buffer
// into the global field gradient: every owned node of every brick is
// written once (no zeroing needed) with the sum of its face slots over the
// bricks in its owner's neighbour list nb[nb_first[o] .. nb_first[o+1]).
// With a group `fg`, only the group's bricks' slots are summed, at the nodes
// the group stores: the first group to reach a node (the group of the lowest
// rank storing it; groups are consecutive rank ranges taken in order) stores
// the sum, later groups add theirs, so the field needs no zeroing either.
size_t face_slots(const int s_n[3]);
cudaError_t launch_face_gather(const BrickDev* bricks, int nbricks, const int* nb_first, const int* nb,
                               long long max_rows, const float4* gface, const int dims[3], float* dvol,
                               cudaStream_t st, const FaceGroup* fg = nullptr);

// Gather layout of a brick (kernels.cu): bytes it needs, and its build from
// the stored nodes.
size_t quad_bytes(int dtype, const int s_n[3]);
cudaError_t launch_build_quad(int dtype, const void* src, const int s_n[3], void* dst, cudaStream_t st);
// Cell gather layout: bytes it needs and its build (eight corners per cell).
size_t cell_bytes(int dtype, const int s_n[3]);
cudaError_t launch_build_cell(int dtype, const void* src, const int s_n[3], void* dst, cudaStream_t st);

// One rank's fragments of one camera, fragment layer `layer` (< P.deep).
cudaError_t launch_read_frags(const FrameParams& P, const Item* items, int n_items, int cam, int rank, int layer,
                              const float4* frag_rgba, const int* frag_key, float4* out_rgba, int* out_key,
                              cudaStream_t st);

}  // namespace dpv
