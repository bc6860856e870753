/*
 * dpv.h -- C ABI of the data-parallel volume renderer (B300, sm_103a).
 *
 * The call shape follows the data-parallel use of ANARI described in
 * "Standardized Data-Parallel Rendering Using ANARI" (arXiv 2407.00179):
 *   - a device is created collaboratively (§3.3);
 *   - each rank defines its own local part of a jointly defined world and
 *     commits it independently (§1, §3.1.2; commit semantics §2.3);
 *   - frame, renderer and camera parameters are globally consistent (§3.1.1);
 *   - rendering is a collaborative, asynchronous call (§3.2, §2.3);
 *   - completion can be waited for or polled (ANARI_WAIT / NO_WAIT, §3.2);
 *   - the final frame is mapped on rank 0 only (§3.1.3);
 *   - the device is released in lock step (§3.2);
 *   - the application tells the device how the data is partitioned (§8.2:
 *     "boundingBox"-style meta parameters): here every rank commits the node
 *     range it owns.
 * All ranks are logical: they are emulated as partitions of one volume on
 * one GPU.  Rank k owns one axis-aligned brick of a structured scalar field
 * and keeps a one-node ghost layer around it.  Rendering ray-marches every
 * brick into one RGBA+key fragment per pixel (emission-absorption, front to
 * back, trilinear samples, 1D RGBA transfer function) and composites the
 * fragments sort-last in per-pixel key order (§2.1, §5.1.1).  An adjoint
 * pass gives gradients of an image loss with respect to the transfer
 * function and the field.
 *
 * Conventions (readings of the paper, which gives no rendering equations):
 *   - nodes: node (i,j,k) sits at world origin + (i,j,k) * spacing; the
 *     volume box is [0, dims-1] in node coordinates;
 *   - a rank owning nodes [lo, hi) per axis owns the region [lo-1/2, hi-1/2]
 *     (clipped to the volume) and stores nodes [lo-1, hi] (clipped);
 *   - samples along a ray sit at t_j = t_enter + (j + 1/2) dt, dt =
 *     step_voxels * spacing, for t_j < t_exit, where [t_enter, t_exit) is the
 *     ray's interval in the volume box clipped to t >= 0; sample j belongs to
 *     the brick whose owned region contains it;
 *   - TF: n RGBA entries at s_i = vmin + i (vmax - vmin)/(n-1), linear
 *     interpolation, clamped outside [vmin, vmax];
 *   - extinction sigma = sigma_max * alpha_TF per world unit, sample opacity
 *     1 - exp(-sigma dt), premultiplied colour accumulation front to back;
 *   - a fragment is (premultiplied RGBA, key = global index of its first
 *     sample); fragments are composited in ascending key order;
 *   - early ray termination, when enabled, is per fragment: a brick stops
 *     once its own opacity exceeds the threshold;
 *   - pinhole cameras, right-handed look-at, rays through pixel centres,
 *     image row 0 at the bottom.
 *
 * Threading and ownership: a device handle must not be used from two host
 * threads at once.  All GPU work is issued asynchronously on the stream
 * given at creation.  Every call returns a status; on failure
 * dpvGetLastError() returns a message for the calling thread.  After a CUDA
 * error the device is poisoned: every later call except dpvRelease returns
 * DPV_ERR_CUDA.
 */
#ifndef DPV_H
#define DPV_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dpv_device_t* dpv_device;

typedef enum {
    DPV_OK = 0,
    DPV_ERR_INVALID_ARG = 1,   /* bad pointer, size, index or parameter */
    DPV_ERR_STATE = 2,         /* call not valid in the current state */
    DPV_ERR_OUT_OF_MEMORY = 3, /* a device or host allocation failed */
    DPV_ERR_CUDA = 4,          /* a CUDA call failed; the device is poisoned */
    DPV_ERR_TIMEOUT = 5,       /* a bounded wait expired */
    DPV_ERR_UNSUPPORTED = 6    /* valid request the library does not handle */
} dpv_status;

typedef enum {
    DPV_F32 = 0,
    DPV_F16 = 1,
    DPV_BF16 = 2,
    DPV_FP8_E4M3 = 3           /* OCP E4M3 (max 448, no infinities) */
} dpv_dtype;

/* One rank's brick.  `data` holds a box of nodes [data_lo, data_lo +
 * data_dims) of the global field, x fastest, in `src_dtype`; it must contain
 * every node the rank stores (owned range plus one ghost node per side,
 * clipped to the volume).  Passing the whole global field (data_lo = 0,
 * data_dims = dims) is allowed: the device extracts what it needs.  The
 * device copies the data (ANARI commit semantics); the caller may free it
 * when dpvCommitBrick returns.  src_dtype must be DPV_F32 (converted to
 * `storage` on the GPU, rounding to nearest even, fp8 saturating) or equal
 * to `storage` (copied).  Stored values are decoded as scale * stored.
 * scale <= 0 selects the default: max|v| / 448 over the stored nodes for
 * DPV_FP8_E4M3 (computed in float32; 1 if all are zero), 1 otherwise. */
typedef struct {
    int owned_lo[3], owned_hi[3];
    dpv_dtype storage;
    float scale;
    dpv_dtype src_dtype;
    const void* data;
    int data_lo[3], data_dims[3];
    int data_on_device;           /* 1: data is a device pointer, 0: host */
} dpv_brick_desc;

/* Pinhole camera: right-handed look-at, vertical field of view in degrees. */
typedef struct {
    float eye[3], center[3], up[3];
    float fovy_deg;
} dpv_camera;

#define DPV_FRAME_ORDER 1          /* also produce the per-pixel order (debug) */
#define DPV_FRAME_STAGED 2         /* stage brick slabs in shared memory instead of
                                      gathering through L1 (same results for float32
                                      bricks; a tuning variant) */
/* Gather layout of the ray-march (identical results in every layout).  By
 * default the device builds, at the next render, the "cell" layout (per cell
 * its 8 corners in one vector: one load per sample, 8x the bricks' device
 * memory) when it fits in half of the free device memory, else the "quad"
 * layout (per cell face the 2x2 corners in one vector: two loads per sample,
 * 4x), and keeps it.  The flags below force a layout; LINEAR takes
 * precedence, then CELL, then QUAD. */
#define DPV_FRAME_LINEAR 4         /* gather the 8 corners from the stored nodes */
#define DPV_FRAME_PERSISTENT 8     /* persistent ray-march: a grid sized to the GPU pulls
                                      work items from a counter in brick-major order (all
                                      cameras' tiles of one brick together).  With
                                      DPV_FRAME_ORDERED: warps pull 32 pixels (a warp's share
                                      of a tile) at a time; the same frame, bit for bit */
#define DPV_FRAME_GRAPH 16         /* replay the frame's launches from a CUDA graph
                                      captured at the first render after a change (not
                                      while profiling is on) */
#define DPV_FRAME_CELL 32          /* the cell layout, whether or not it fits */
#define DPV_FRAME_QUAD 64          /* the quad layout */
#define DPV_FRAME_ORDERED 256      /* visibility-ordered march with global early termination:
                                      each ray marches the bricks it crosses front to back
                                      (entry sample order), carrying the accumulated colour
                                      and transmittance from brick to brick, and stops once
                                      the accumulated opacity passes ert_threshold; bricks
                                      behind are not marched.  Writes the frame directly (no
                                      fragments, no sort-last composite).  No backward
                                      (DPV_ERR_UNSUPPORTED); not with DPV_FRAME_STAGED or
                                      DPV_FRAME_ISO. */
#define DPV_FRAME_SKIP 512         /* empty-space skipping in the forward march (sort-last
                                      or ordered): samples inside a macro-cell (8^3 cells)
                                      whose value range reaches only TF entries of opacity
                                      0 are not evaluated (their alpha is exactly 0, so the
                                      frame is bit-identical); the macro-cell ranges are
                                      built once per committed brick, their transparency
                                      per render.  Sample counts then count the evaluated
                                      samples.  The backward replays every sample. */
#define DPV_FRAME_DEEP 1024       /* deep fragments: empty-space skipping (implied) splits
                                      a brick's ray segment at its transparent macro-cells,
                                      each run of evaluated samples becoming its own
                                      fragment (key = the run's first sample index); up to
                                      DPV_DEEP_MAX per brick and pixel, later runs continue
                                      the last one.  The compositor sorts the variable
                                      count per pixel (§2.1, §5.1.1: several fragments per
                                      pixel from one rank).  Early termination stays on the
                                      brick's accumulated opacity.  Forward only (the
                                      adjoint returns DPV_ERR_UNSUPPORTED); not with
                                      STAGED, ISO or ORDERED.  The order image then has
                                      num_ranks x DPV_DEEP_MAX entries per pixel, one brick
                                      id per fragment. */
#define DPV_DEEP_MAX 4
#define DPV_FRAME_SHADOW 2048     /* volumetric shadows by ray forwarding: every sample's
                                      emission is scaled by k_a + (1 - k_a) T_light, T_light
                                      the transmittance of a shadow ray toward the light of
                                      dpvSetLight, sampled at p + (i + 1/2) h L inside the
                                      volume box.  Each brick's samples spawn one wave-front
                                      of shadow rays; in num_ranks rounds every brick marches
                                      every wave-front through the samples it owns (a ring
                                      exchange of full wave-fronts, §2.3), then the shading
                                      march writes ordinary fragments.  Opacity, keys, depth
                                      and the composite are those of the sort-last frame.
                                      Forward only; not with STAGED, ISO, ORDERED, SKIP or
                                      DEEP.  Needs dpvSetLight. */
#define DPV_FRAME_ISO 128          /* iso-surface fragments instead of volume rendering
                                      (the paper's z-composited opaque surfaces, §7):
                                      each brick reports the first sample pair (j-1, j)
                                      of the ray, j its own, across which [s >= iso_value]
                                      changes (it evaluates s_{j-1} in its ghost layer);
                                      the surface point is interpolated linearly between
                                      the two samples; colour = TF rgb(iso_value) x
                                      (0.25 + 0.75 |N.d| / (|N||d|)), N the gradient of
                                      the trilinear interpolant, alpha 1; the composite
                                      keeps the nearest fragment (smallest key) and its
                                      interpolated depth.  No hit: (0,0,0,0), depth +inf.
                                      No backward (DPV_ERR_UNSUPPORTED), not with
                                      DPV_FRAME_STAGED. */

/* Frame parameters, identical on all ranks (§3.1.1).  Every camera renders
 * a width x height image.  tile_w/tile_h: pixels per work item (multiples
 * of 8 and 4; 0 = autotuned default).  ert_threshold <= 0 or >= 1 disables
 * early termination.  iso_value: the level of DPV_FRAME_ISO. */
typedef struct {
    int width, height;
    float step_voxels;
    float sigma_max;
    float ert_threshold;
    int tile_w, tile_h;
    int flags;
    float iso_value;
} dpv_frame_desc;

/* Pipeline stages timed when profiling is on (dpvSetProfiling). */
typedef enum {
    DPV_STAGE_CULL = 0,           /* camera setup, culling, work list */
    DPV_STAGE_MARCH = 1,          /* brick ray-march (forward) */
    DPV_STAGE_COMPOSITE = 2,      /* sort-last compositor (forward) */
    DPV_STAGE_COMPOSITE_BWD = 3,  /* compositor adjoint */
    DPV_STAGE_MARCH_BWD = 4,      /* ray-march adjoint (the replay launches) */
    DPV_STAGE_FACE = 5,           /* face adjoint buffer of the field gradient:
                                     clears and gathers into the field */
    DPV_NUM_STAGES = 6
} dpv_stage;

/* Counters.  samples_* and error_flags are those of the most recent
 * dpvRenderFrame / dpvBackward.  stage_ms / stage_calls: device time of each
 * stage, measured with CUDA events on the device stream around its kernels,
 * summed over all renders since the last dpvResetStats while profiling was
 * on.  kernel_launches: kernels this device launched since the last reset. */
typedef struct {
    uint64_t samples_forward;     /* samples evaluated by the ray-march */
    uint64_t samples_backward;    /* samples replayed by the adjoint march */
    uint64_t work_items;          /* (camera, brick, tile) items marched */
    uint64_t fragment_bytes;      /* device bytes held by the fragment pool */
    uint32_t error_flags;         /* device-side error bits (0 = none) */
    uint32_t max_fragments;       /* most fragments listed for one tile */
    double stage_ms[DPV_NUM_STAGES];
    uint32_t stage_calls[DPV_NUM_STAGES];
    uint64_t kernel_launches;
    uint64_t graph_launches;      /* frames replayed from a CUDA graph since the reset */
    uint64_t samples_shadow;      /* shadow samples evaluated (DPV_FRAME_SHADOW) */
} dpv_stats;

/* Create a device for `num_ranks` logical ranks (1..255) on CUDA device
 * `cuda_device`, issuing all work on `cuda_stream` (a cudaStream_t; NULL =
 * the legacy default stream).  The stream must outlive the device.
 * Paper: every rank creates the data-parallel device together (§3.3, §2.3);
 * here one handle stands for all logical ranks.  *out is written only on
 * success; DPV_ERR_INVALID_ARG for a bad rank count, device or NULL out,
 * DPV_ERR_CUDA if the device cannot be set up. */
dpv_status dpvCreateDevice(int num_ranks, int cuda_device, void* cuda_stream, dpv_device* out);

/* Global node grid: dims[a] >= 2 nodes per axis, world origin of node 0 and
 * isotropic spacing > 0.  Must be set before bricks are committed; setting
 * it again discards all bricks.  Paper: the world is one jointly defined
 * entity whose parts the ranks own (§1, §3.1.1 ANARIWorld is global); the
 * grid is the frame of reference of every rank's part.  Host arrays, read
 * during the call.  DPV_ERR_INVALID_ARG for dims < 2 or spacing <= 0. */
dpv_status dpvSetVolumeGeometry(dpv_device dev, const int dims[3], const float origin[3], float spacing);

/* Commit rank `rank`'s brick (copies, see dpv_brick_desc).  Ranks commit
 * independently, in any order (§3.1.2).  A brick may hold at most 2^31 - 1
 * stored nodes.  All ranks of a device must use the same storage dtype.
 * Blocks the host until the copy has been issued; with host data it returns
 * after the host buffer has been read. */
dpv_status dpvCommitBrick(dpv_device dev, int rank, const dpv_brick_desc* desc);

/* Transfer function: n (2..4096) RGBA float entries, x fastest, on the host
 * (on_device = 0) or the device; values over [vmin, vmax], vmax > vmin.
 * Copied; visible to the next render.  A host table is copied into one of
 * two pinned staging buffers and uploaded on the device stream: the
 * caller's buffer may be reused at return and the call does not wait for
 * the device (only for the upload issued two calls earlier).  A device
 * table is copied on the device stream.  Paper: renderer and camera
 * parameters are identical on every rank (§3.1.1); the table is the
 * renderer's classification.  `on_device` has no counterpart in the call
 * shape of the paper: it says where `rgba` lives so a render loop can
 * feed a table it keeps on the GPU.  DPV_ERR_INVALID_ARG for NULL rgba, n
 * out of range or vmax <= vmin. */
dpv_status dpvSetTransferFunction(dpv_device dev, const float* rgba, int n, float vmin, float vmax, int on_device);

/* Directional light for DPV_FRAME_SHADOW: direction toward the light (any
 * non-zero length; normalised here), shadow sample spacing h in voxels
 * (1/64 .. 64), ambient term k_a in [0, 1] (1: no shadows).  Visible to the
 * next render; DPV_ERR_INVALID_ARG otherwise.  Paper: shadows are the
 * global effect the paper says compositing cannot give and ray forwarding
 * between ranks can (§2.2, §7); the light is a renderer parameter and so
 * globally consistent (§3.1.1). */
dpv_status dpvSetLight(dpv_device dev, const float direction[3], float step_voxels, float ambient);

/* Cameras (host array of n >= 1, read during the call).  Every render
 * produces one image each.  Paper: the camera is globally consistent, set
 * identically on every rank (§3.1.1); several cameras form one batch.
 * DPV_ERR_INVALID_ARG for NULL, n < 1, fovy outside (0, 180), eye equal to
 * center or up parallel to the view direction. */
dpv_status dpvSetCameras(dpv_device dev, const dpv_camera* cams, int n);

/* Frame parameters (host struct, read during the call).  Paper: the frame
 * is a global object whose parameters match on every rank (§3.1.1).
 * DPV_ERR_INVALID_ARG for a non-positive size or step, a tile that is not
 * a multiple of 8 x 4 or above 256 pixels, or conflicting flags. */
dpv_status dpvSetFrame(dpv_device dev, const dpv_frame_desc* desc);

/* Render one frame for every camera: cull, brick ray-march and sort-last
 * composite, asynchronously on the device stream (§3.2: collaborative).
 * Every rank must have committed a brick, and the owned ranges must tile
 * the volume exactly, else DPV_ERR_STATE / DPV_ERR_INVALID_ARG.  The first
 * render after a change of geometry, bricks, cameras or frame size blocks
 * while it sizes the fragment pool. */
dpv_status dpvRenderFrame(dpv_device dev);

/* Frame completion: wait = 1 blocks until the last render has finished
 * (ANARI_WAIT); wait = 0 only polls (ANARI_NO_WAIT).  *ready = 1 when done.
 * Paper: the property query of a frame synchronises with WAIT and may
 * return at once with NO_WAIT (§3.2).  DPV_ERR_INVALID_ARG for NULL ready;
 * DPV_ERR_CUDA if the render failed on the device. */
dpv_status dpvFrameReady(dpv_device dev, int wait, int* ready);

/* Device pointers to camera `camera`'s composited frame: rgba = height x
 * width x 4 floats (premultiplied, row 0 at the bottom), depth = height x
 * width floats (t of the first sample of the first fragment with non-zero
 * opacity, +inf if none).  Device-owned, valid until the next render or
 * release; read them on the device stream or after dpvFrameReady.  Paper:
 * the final frame is mapped on rank 0 with the ordinary map call (§3.1.3);
 * here the one device holds it.  Unmap releases nothing (the buffers are
 * the device's) and only checks the camera index.  DPV_ERR_STATE before
 * the first render, DPV_ERR_INVALID_ARG for a camera out of range. */
dpv_status dpvMapFrame(dpv_device dev, int camera, const float** rgba, const float** depth);
dpv_status dpvUnmapFrame(dpv_device dev, int camera);

/* Copy camera `camera`'s frame into caller buffers (device or host
 * pointers; either may be NULL), ordered on the device stream.  Returns
 * after the copy has been issued (host destinations: after it completed).
 * Paper: the final frame is delivered on rank 0 (§3.1.3); this is the map
 * followed by a copy.  DPV_ERR_STATE / DPV_ERR_INVALID_ARG as dpvMapFrame. */
dpv_status dpvCopyFrame(dpv_device dev, int camera, float* rgba, float* depth);

/* Asynchronous copy of camera `camera`'s frame (camera = -1: every camera's,
 * in camera order, contiguous) into caller buffers (host or device; either
 * pointer may be NULL).  The frame is first copied on the device stream into
 * one of two device staging slots; a separate copy stream then moves it to
 * the destination while the device stream goes on with the next render.
 * Returns at once.  The destination is complete after dpvCopyWait.  A third
 * copy in flight waits on the device stream until the slot it reuses has
 * drained.  Destinations in pageable host memory copy synchronously with
 * respect to the host (CUDA's rule); pinned memory overlaps.  Paper: frame
 * delivery on rank 0 (§3.1.3) under ANARI's asynchronous rendering (§3.2);
 * overlapping the copy with the next render has no counterpart there. */
dpv_status dpvCopyFrameAsync(dpv_device dev, int camera, float* rgba, float* depth);

/* Block until every copy dpvCopyFrameAsync issued has completed (the wait
 * of the asynchronous delivery above; no counterpart in the paper). */
dpv_status dpvCopyWait(dpv_device dev);

/* Map rank `rank`'s fragments of camera `camera` from the last render.
 * *frag points to a device-owned block: height x width float4 (the
 * fragments' premultiplied RGBA, x fastest, row 0 at the bottom), followed
 * at byte offset 16 x width x height by height x width int32 keys (the
 * global index of the fragment's first sample; 2^31 - 1 = empty, also for
 * pixels the rank was culled from).  The block is filled on the device
 * stream by this call (read it on that stream or after dpvFrameReady) and
 * stays allocated until dpvUnmapFragments for the same camera and rank, or
 * release; a later render does not refresh it (map again).  Layer 0 of a
 * DPV_FRAME_DEEP frame (dpvReadDeepFragments reads the others).  Paper:
 * each rank's fragment image is the compositor's per-rank input (§5.1.1),
 * and mapping gives read access to device-held pixels (§3.1.3).
 * DPV_ERR_STATE before the first render, DPV_ERR_INVALID_ARG for a camera
 * or rank out of range or NULL frag, DPV_ERR_OUT_OF_MEMORY if the block
 * cannot be allocated. */
dpv_status dpvMapFragments(dpv_device dev, int camera, int rank, const void** frag);

/* Release the block dpvMapFragments returned for (camera, rank); waits for
 * the device stream first.  Paper: the unmap that ends a map (§3.1.3).
 * DPV_ERR_STATE if that pair is not mapped. */
dpv_status dpvUnmapFragments(dpv_device dev, int camera, int rank);

/* Debug/test: write rank `rank`'s fragments for camera `camera` into caller
 * device buffers rgba (height x width x 4, premultiplied) and key (height x
 * width int32; 2^31 - 1 = empty, also for pixels the rank was culled from);
 * the copy form of dpvMapFragments (§5.1.1: a rank's fragments).
 * DPV_ERR_STATE before the first render, DPV_ERR_INVALID_ARG for a camera
 * or rank out of range or a NULL buffer. */
dpv_status dpvReadFragments(dpv_device dev, int camera, int rank, float* rgba, int32_t* key);

/* Debug/test: as dpvReadFragments, for fragment layer `layer` of a frame
 * rendered with DPV_FRAME_DEEP (0 <= layer < DPV_DEEP_MAX; layers past a
 * pixel's fragment count read as empty).  Without DPV_FRAME_DEEP only layer 0
 * exists.  Paper: several fragments per pixel from one rank, the general
 * input of the compositor (§2.1, §5.1.1).  DPV_ERR_INVALID_ARG for a layer
 * out of range. */
dpv_status dpvReadDeepFragments(dpv_device dev, int camera, int rank, int layer, float* rgba, int32_t* key);

/* Debug/test: copy rank `rank`'s stored nodes (owned + ghost box, x
 * fastest, in the storage format) to the caller's device buffer `dst` (NULL
 * to skip) and return the box and the rank's decode scale (synchronises the
 * device stream).  stored_lo/stored_dims/scale may be NULL.  Paper: the
 * rank's locally defined data (§3.1.2) as committed, ghost layer included
 * (§1).  DPV_ERR_STATE if the rank has not committed. */
dpv_status dpvReadBrick(dpv_device dev, int rank, void* dst, int stored_lo[3], int stored_dims[3], float* scale);

/* Debug/test (needs DPV_FRAME_ORDER): device pointer to camera `camera`'s
 * order image: height x width x stride bytes, the ranks of the pixel's
 * non-empty fragments front to back, then 0xFF.  Paper: the compositor
 * sorts each pixel's fragments by depth (§5.1.1); this is that order.
 * DPV_ERR_STATE without DPV_FRAME_ORDER, DPV_ERR_INVALID_ARG for a camera
 * out of range. */
dpv_status dpvMapOrder(dpv_device dev, int camera, const uint8_t** order, int* stride);

/* Adjoint of the last render (the differentiable form: no counterpart in
 * the paper, whose renderer is forward only; the operations it inverts are
 * the ray-march of one rank's part and the sort-last composite, §2.1,
 * §5.1.1).  dL_drgba: device array cameras x height x
 * width x 4 floats (gradient of the loss with respect to the composited
 * premultiplied RGBA).  dL_dtf: device array n x 4 doubles, overwritten with
 * the gradient with respect to the TF entries.  dL_dvol: device array of the
 * global field's size (x fastest) of floats, overwritten with the gradient
 * with respect to the field values (a ghost copy's share goes to its global
 * node), or NULL.  Both outputs are zeroed by the call.  Uses the fragments
 * of the last render: call it before the next render.  Asynchronous on the
 * device stream.  The field gradient goes through a face adjoint buffer
 * (one float4 per cell face of every brick) that the first call allocates,
 * up to half of the free device memory, and keeps until release (it is not
 * tried again until the bricks' sizes change). Where not all bricks fit at
 * once, they are replayed in groups of consecutive ranks, two launches per
 * group. Where not even one brick fits, the field gradient goes with scalar
 * atomics straight into dL_dvol.  Where a brick's slots are far larger
 * than L2 (over 8x), each thread sums the samples it takes in one cell in
 * registers before reducing into the buffer.  Environment (tests):
 * DPV_FACE_GRAD=0 takes the scalar atomics; DPV_FACE_GROUP=n puts at most n
 * bricks in a group; DPV_FACE_RUNS=0/1 turns the per-cell sums off or on. */
dpv_status dpvBackward(dpv_device dev, const float* dL_drgba, double* dL_dtf, float* dL_dvol);

/* Counters (synchronises the device stream).  Tracing has no counterpart
 * in the paper.  DPV_ERR_INVALID_ARG for NULL out. */
dpv_status dpvGetStats(dpv_device dev, dpv_stats* out);

/* Result of dpvAutotune. */
typedef struct {
    int tile_w, tile_h;   /* chosen tile */
    int flags;            /* chosen layout (DPV_FRAME_CELL / QUAD / LINEAR) and
                             DPV_FRAME_PERSISTENT bits */
    float ms;             /* mean device time of one frame with the choice */
    int candidates;       /* configurations timed */
} dpv_tune_result;

/* Autotuner: time candidate launch configurations of the current scene --
 * tile shape (16x16, 32x8, 8x32, 64x4) x gather layout (quad, linear) x
 * schedule (one CTA per work item, persistent brick-major) -- rendering
 * `frames` frames each after one warm-up frame, and keep the fastest in the
 * device's frame parameters (other flags are kept).  Needs a renderable
 * device; blocks the host until done; the last rendered frame is the best
 * candidate's.  Launch forms have no counterpart in the paper (its device
 * implementation is left to the vendor, §3.2). */
dpv_status dpvAutotune(dpv_device dev, int frames, dpv_tune_result* out);

/* Clear the accumulated stage times and the launch count (tracing: no
 * counterpart in the paper). */
dpv_status dpvResetStats(dpv_device dev);

/* Turn per-stage CUDA-event timing on (1) or off (0) (tracing: no
 * counterpart in the paper). */
dpv_status dpvSetProfiling(dpv_device dev, int enable);

/* One rank's brick for dpvRenderNoAlloc: a device pointer to the nodes the
 * rank stores (its owned range plus one ghost node per side, clipped to the
 * volume; x fastest) in the scene's storage format, decoded as
 * scale * stored (scale <= 0 means 1).  Caller-owned. */
typedef struct {
    int owned_lo[3], owned_hi[3];
    const void* data;
    float scale;
} dpv_noalloc_brick;

/* Everything dpvRenderNoAlloc reads: the grid, the ranks' bricks (host
 * array of num_ranks entries, all in `storage`, read during the call), and
 * the transfer function (device pointer, 16-byte aligned, tf_n RGBA
 * floats). */
typedef struct {
    int dims[3];
    float origin[3];
    float spacing;
    int num_ranks;
    const dpv_noalloc_brick* bricks;
    dpv_dtype storage;
    const float* tf_rgba;
    int tf_n;
    float vmin, vmax;
} dpv_noalloc_scene;

/* Allocation-free render (the paper has no counterpart: this entry point is
 * for callers that cannot allocate device memory -- applications whose
 * device memory belongs to their own pool or a framework's caching
 * allocator, and render loops that cannot afford the device-wide
 * synchronisation of cudaMalloc and cudaFree).
 * Renders one camera exactly as dpvRenderFrame does (cull, brick ray-march,
 * sort-last composite) into the caller's device buffers rgba (height x width
 * x 4 floats, 16-byte aligned) and depth (height x width floats), on
 * `cuda_stream`, on the current CUDA device.  It calls no cudaMalloc or
 * cudaFree: its intermediate buffers live in one fixed 64 MiB device array
 * that the library holds on every GPU it is loaded on until the process
 * exits.  A frame needs about width x height x (80 + 20 x num_ranks) bytes
 * of it (e.g. 512 x 512 with 8 ranks); larger requests fail with
 * DPV_ERR_INVALID_ARG.  The first call on a device looks up the array's
 * device address (cudaGetSymbolAddress) and keeps it.  Every call reuses the
 * same array, so calls that overlap on the GPU -- on different streams or
 * from different host threads -- race and must be serialised by the caller.
 * It marches the linear gather layout and ignores the layout, staged,
 * persistent and graph bits of frame->flags; DPV_FRAME_ISO,
 * DPV_FRAME_ORDERED, DPV_FRAME_SKIP, DPV_FRAME_DEEP, DPV_FRAME_SHADOW and
 * DPV_FRAME_ORDER return DPV_ERR_UNSUPPORTED (they need device state).
 * Cameras are checked as dpvSetCameras checks them.  Its small host tables
 * (brick table, scales, camera) travel to the device as kernel parameters,
 * so the call reads none of the caller's host memory after it returns.
 * Asynchronous: returns once the work is queued. */
dpv_status dpvRenderNoAlloc(const dpv_noalloc_scene* scene, const dpv_camera* camera, const dpv_frame_desc* frame,
                            float* rgba, float* depth, void* cuda_stream);

/* Message of the last failed call on this host thread ("" if none).  Error
 * reporting through status codes and messages has no counterpart in the
 * paper. */
const char* dpvGetLastError(void);

/* Release the device and all its memory (§3.2: lock step).  NULL is OK. */
dpv_status dpvRelease(dpv_device dev);

#ifdef __cplusplus
}
#endif

#endif /* DPV_H */
