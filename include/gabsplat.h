/*
 * gabsplat.h -- C ABI of the B300 (sm_103a) 3D Gabor splatting rasterizer.
 *
 * Method: "3DGabSplat: 3D Gabor Splatting for Frequency-adaptive Radiance Field Rendering"
 * (arXiv 2508.05343).  A primitive k has mean mu_k, covariance Sigma_k = R_k S_k S_k^T R_k^T,
 * opacity o_k, SH colour coefficients c_k and F = K Gabor components (f_{k,i}, w_{k,i})
 * (Sec. 3.1, Sec. 3.2.1 Eq. 5).  Rendering projects the envelope with the EWA map
 * J W Sigma W^T J^T (Sec. 3.1, Eq. 2), each frequency with ((JW)^-1)^T f (Sec. 3.3.1, Eq. 7) and
 * z-integrates it to f2D (Sec. 3.3.2, Eq. 8), bins the splats into 16x16 tiles sorted by depth
 * and alpha-composites them front to back (Sec. 3.3.3, Eq. 10).
 *
 * Conventions shared by every call
 * --------------------------------
 *  - All pointers named "device" are CUDA device pointers; the library never allocates or frees
 *    device memory and never synchronises, except gabsplat_device_status, which copies the
 *    workspace header to the host and synchronises the given stream.  The caller owns every
 *    buffer, including the workspace.  Every call is asynchronous on `stream` (a cudaStream_t;
 *    NULL = the legacy default stream).
 *  - Host-detectable errors (null pointer, n < 0, K > GS_MAX_K, bad image size, workspace too
 *    small) return immediately without launching anything.  Errors found on the device (pair
 *    capacity exceeded, a bounded spin that timed out, non-finite projected values) are written
 *    to a status word inside the workspace; every later stage of the same frame then does
 *    nothing, and gabsplat_device_status() reports the error.
 *  - Inputs are activated values: positive scales, opacity and weights in [0, 1).  Quaternions
 *    (w, x, y, z) may have any non-zero norm; they are normalised on the device and gradients
 *    flow through the normalisation.
 *  - Images are planar float32: rgb [3][height][width], transmittance [height][width].
 *    Pixel (i, j) samples the point (i + 0.5, j + 0.5).
 */
#ifndef GABSPLAT_H
#define GABSPLAT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define GS_TILE 16          /* tile edge in pixels (fixed) */
#define GS_MAX_K 8          /* largest number of Gabor components per primitive */
#define GS_MAX_SH_DEGREE 3  /* largest spherical-harmonics degree */
#define GS_MAX_VIEWS 16     /* largest number of views in one batched frame */

typedef struct CUstream_st* gs_stream; /* identical to cudaStream_t */

typedef enum {
  GS_OK = 0,
  GS_ERR_INVALID_ARG = 1, /* host-side argument check failed */
  GS_ERR_CAPACITY = 2,    /* more (tile, primitive) pairs than the workspace holds */
  GS_ERR_TIMEOUT = 3,     /* a bounded device-side wait gave up */
  GS_ERR_CUDA = 4,        /* a CUDA launch or copy failed */
  GS_ERR_NONFINITE = 5,   /* a projected mean or covariance was not finite */
  GS_ERR_WORKSPACE = 6    /* workspace pointer/size does not match the frame description */
} gs_status;

typedef enum { GS_F32 = 0, GS_BF16 = 1 } gs_dtype;
typedef enum { GS_LOSS_L1 = 0, GS_LOSS_L2 = 1 } gs_loss_kind;

/* Primitive attributes (Sec. 3.1 and Sec. 3.2.1), all device pointers, row-major.
 *   means   [n][3] float32          world-space mu_k
 *   scales  [n][3] float32 (> 0)    diagonal of S_k
 *   quats   [n][4] float32          rotation R_k as quaternion (w, x, y, z), any norm > 0,
 *                                   16-byte aligned
 *   opacity [n]    float32 in [0,1)
 *   sh      [n][(sh_degree+1)^2][3] float32 or bf16 (storage)   SH colour coefficients c_k
 *   freqs   [n][K][3]   float32 or bf16    world-frame frequencies f_{k,i}, cycles per unit
 *   weights [n][K]      float32 or bf16    Gabor weights w_{k,i} in [0, 1)
 * freqs/weights may be NULL when K == 0.  storage applies to sh, freqs and weights together;
 * BF16 values are widened to float32 on load and all arithmetic is float32/float64. */
typedef struct {
  int n, K, sh_degree, storage;
  const float* means;
  const float* scales;
  const float* quats;
  const float* opacity;
  const void* sh;
  const void* freqs;
  const void* weights;
} gs_prims;

/* Pinhole camera.  R (row-major 3x3) and t map world to camera space (x right, y down,
 * z forward): x_cam = R x_world + t.  Image coordinates: u = fx x/z + cx, v = fy y/z + cy.
 * Primitives with camera depth z <= znear or z > zfar are culled. */
typedef struct {
  float R[9];
  float t[3];
  float fx, fy, cx, cy;
  int width, height;
  float znear, zfar;
} gs_camera;

/* Rasterizer constants of the tile rasterizer the paper adopts (Sec. 3.3.3):
 * eps2d is added to the diagonal of the 2D covariance, alpha = min(alpha_max, o Gabor2D(x)),
 * pairs with alpha < alpha_min are skipped, compositing stops before the pair whose
 * T (1 - alpha) would drop below T_min, and bg is added with the final transmittance.
 * Defaults: 0.3, 0.99, 1/255, 1e-4, (0,0,0).  flags: 0 (the method as the paper renders it) or
 * GS_FLAG_Z_ATTENUATION: the variant that keeps the z-integration constant C2 of supplement A.2,
 * so the 2D filter bank is (1 - sum w_i) + sum w_i C2_i cos(2 pi f2D_i . d) with
 * C2_i = exp(-2 pi^2 f_proj,z,i^2 / S_22), S the inverse of the ray-space covariance J W Sigma
 * W^T J^T (undilated).  Other bits are rejected. */
#define GS_FLAG_Z_ATTENUATION 1u
typedef struct {
  float eps2d, alpha_max, alpha_min, T_min;
  float bg[3];
  unsigned flags;
} gs_config;

/* Sizes of one frame and the caller-owned device workspace that holds its state between the
 * calls (projected records, (tile, depth rank) pairs, tile ranges, per-pixel transmittance and last
 * contributor).  One frame = one view of one scene.  The same frame description and
 * workspace must be passed to every stage of that frame; the stages of two frames that share
 * a workspace must not overlap on the device. */
typedef struct {
  int n, K, sh_degree, width, height;
  int storage;                      /* gs_dtype of sh/freqs/weights; must equal gs_prims.storage */
  unsigned long long pair_capacity; /* most (tile, primitive) pairs the workspace can hold */
  void* ws;                         /* device pointer, 256-byte aligned */
  size_t ws_bytes;
} gs_frame;

/* Gradients (float32, device, same shapes as gs_prims; overwritten, not accumulated).
 * means2d [n][2] receives dL/d(projected mean) for density-control statistics; any pointer
 * may be NULL to skip that output. */
typedef struct {
  float* means;
  float* scales;
  float* quats;
  float* opacity;
  float* sh;
  float* freqs;
  float* weights;
  float* means2d;
} gs_prim_grads;

/* Device pointers into a workspace, for inspection and tests (valid after the stage that
 * writes them).  Primitives that reach at least one tile are "active"; they are numbered by depth
 * rank r = 0 .. n_active - 1 (camera depth ascending, ties by primitive index), and order[r] is the
 * primitive of rank r.  records: [n_active][record_floats], row r for the primitive of rank r, the
 * projected 2D primitive laid out as
 *   {mu_x, mu_y, conic_a, conic_b, conic_c, opacity, 1 - sum w, depth, r, g, b, 0,
 *    f2D_0x, f2D_0y, ..., f2D_(K-1)y, w_0 .. w_(K-1), 0 padding to a multiple of 4}
 * where the 2D Gaussian is exp(-(a dx^2 + c dy^2)/2 - b dx dy) and f2D is in cycles per pixel.
 * touched [n] uint32 kept tiles per primitive (by primitive index); offsets [n_active] uint32 first
 * pair position of each rank; keys [pairs] uint64 = tile << 32 | depth rank (sorted: by tile, then
 * rank, so each tile's pairs are in depth order; unsorted: emission order); ranges [tiles][2] uint32
 * [start, end);
 * T_final [H][W] float32; n_contrib [H][W] uint32 (1-based position in the tile's list of
 * the last composited pair); the per-pixel work counters, written only by
 * gabsplat_render_fwd_stats: n_eval [H][W] uint32 pairs the forward pass evaluated at the pixel
 * (its tile's list length, or up to the pair that ended compositing); n_reach [H][W] uint32 of those,
 * pairs whose envelope passed o G >= alpha_min; n_comp [H][W] uint32 pairs composited; grad2d
 * [n_active][grad2d_floats] float32 by depth rank
 *   {d mu_x, d mu_y, d a, d b, d c, d opacity, d r, d g, d b, d f2D (2K), d (cosine weight) (K),
 *    d (1 - sum w), 0 pad}: the filter bank (1 - sum w) + sum w'_i cos(.) is differentiated in its
 *    two weight terms separately (w' = w, or w C2 in the z-attenuation variant, whose records hold
 *    w' in the weight slots). */
typedef struct {
  float* records;
  unsigned* touched;
  unsigned* offsets;
  unsigned* order;
  unsigned n_active;
  unsigned long long* keys_sorted;
  unsigned long long* keys_unsorted;
  unsigned* ranges;
  float* T_final;
  unsigned* n_contrib;
  unsigned* n_eval;
  unsigned* n_reach;
  unsigned* n_comp;
  float* grad2d;
  int record_floats;
  int grad2d_floats;
  int tiles_x, tiles_y;
} gs_ws_views;

/* Bytes of device workspace a frame needs.  Returns 0 if the sizes are invalid. */
size_t gabsplat_workspace_size(int n, int K, int sh_degree, int width, int height,
                               unsigned long long pair_capacity);

/* Zero-fills the workspace (asynchronously on `stream`).  Required once after the workspace is
 * allocated (or allocate it zero-filled): the radix sort's passes tag their look-back words with
 * a per-frame epoch, and a zeroed word is never mistaken for a published one. */
gs_status gabsplat_workspace_init(const gs_frame* frame, gs_stream stream);

/* Stage 1, per-primitive projection (Sec. 3.1 Eq. 2, Sec. 3.3.1 Eq. 7, Sec. 3.3.2 Eq. 8):
 * culls, projects mean and covariance (float64 determinant and conic), evaluates SH colour
 * at the viewing direction, splats the K frequencies to f2D, and writes one 2D record and
 * the number of touched tiles per primitive into the workspace.  The config given here applies
 * to the whole frame (render and backward). */
gs_status gabsplat_preprocess(const gs_frame* frame, const gs_prims* prims, const gs_camera* cam,
                              const gs_config* cfg, gs_stream stream);

/* Stage 2, tile binning and depth sort (Sec. 3.1, "sorted by depth"; Sec. 3.3.3).  Inside the
 * preprocess call: the active primitives are sorted by camera depth (a stable radix sort of their
 * depth keys, so equal depths keep primitive order), the kept-tile counts are scanned in that
 * order, and one (tile << 32 | depth rank) pair is emitted per kept tile, in rank order.  This
 * call sorts the pairs by tile with a stable least-significant-digit radix sort of the tile bits,
 * which leaves each tile's pairs in (depth, primitive) order, and writes per-tile [start, end)
 * ranges.  The pair count stays on the device.  GS_ERR_CAPACITY (device status) if it exceeds
 * frame->pair_capacity; gabsplat_device_status() then reports the needed count. */
gs_status gabsplat_bin_sort(const gs_frame* frame, gs_stream stream);

/* Stage 3, front-to-back alpha compositing of the 2D Gabor primitives (Sec. 3.3.2 Eq. 9 and
 * Sec. 3.3.3 Eq. 10) with the constants of the gs_config given to gabsplat_preprocess.
 * out_rgb [3][H][W] (device, required) and out_T [H][W] (device, may be NULL).  Keeps the final
 * transmittance and the last contributor per pixel in the workspace for the backward pass. */
gs_status gabsplat_render_fwd(const gs_frame* frame, float* out_rgb, float* out_T, gs_stream stream);

/* gabsplat_render_fwd that also writes the per-pixel work counters (n_eval, n_reach, n_comp of
 * gabsplat_workspace_views: pairs evaluated, reached by the envelope, composited), for work
 * accounting and tests.  The image, the transmittance, the last contributor and the state the
 * backward pass reads are the same; the counters cost the forward about 7% of its time, so
 * gabsplat_render_fwd leaves them as they were.  The paper has no counterpart. */
gs_status gabsplat_render_fwd_stats(const gs_frame* frame, float* out_rgb, float* out_T, gs_stream stream);

/* Stage 3 for frames that will not be differentiated (rendering only): the same images and
 * per-pixel state as gabsplat_render_fwd, without recording, per warp of 64 pixels, which pairs
 * its pixels composited (the bits the backward pass walks), which makes it faster.
 * gabsplat_render_bwd_2d after it (with no gabsplat_render_fwd of the same frame) sets
 * GS_ERR_INVALID_ARG in the device status. */
gs_status gabsplat_render_fwd_only(const gs_frame* frame, float* out_rgb, float* out_T, gs_stream stream);

/* Frequency maps (the visualisation of Sec. 4: the weighted Gabor frequencies of the primitives
 * blended into the image): the compositing of stage 3 with each primitive's colour replaced by
 * three frequency features of its splatted components (Eq. 8) and no background:
 *   out_map[0] = sum over pairs of alpha T (sum_i w_i |f2D_i|),
 *   out_map[1] = ... (sum_i w_i |f2D_i,x|),  out_map[2] = ... (sum_i w_i |f2D_i,y|),
 * f2D in cycles per pixel.  out_map [3][H][W] float32, device, required.  Runs after
 * gabsplat_bin_sort like gabsplat_render_fwd (before or after it: both make the same per-pixel
 * decisions and leave the same per-pixel state for the backward pass).  All zero for K = 0. */
gs_status gabsplat_render_freq_map(const gs_frame* frame, float* out_map, gs_stream stream);

/* Stage 4, reverse-order backward pass of the differentiable rasterizer (Sec. 3.3.3, trained by
 * the photometric loss of Sec. 3.4.1).  Given dL/d(rgb) [3][H][W] (device), walks each pixel's
 * pairs back to front from its last contributor, recomputing transmittance by division instead of
 * storing per-pair state, accumulates per-primitive 2D gradients, and chains them to every
 * attribute in gs_prim_grads.  Uses the primitives and camera given to gabsplat_preprocess for
 * this frame (their buffers must still hold the same values). */
gs_status gabsplat_render_bwd(const gs_frame* frame, const float* dL_drgb, const gs_prim_grads* grads,
                              gs_stream stream);

/* The two halves of gabsplat_render_bwd, callable separately (e.g. to time them):
 * gabsplat_render_bwd_2d clears grad2d (workspace), then accumulates the per-primitive 2D gradients
 * from dL/d(rgb); gabsplat_preprocess_bwd zero-fills every array of gs_prim_grads, then chains
 * grad2d to the attributes of the primitives that reach a tile. */
gs_status gabsplat_render_bwd_2d(const gs_frame* frame, const float* dL_drgb, gs_stream stream);
gs_status gabsplat_preprocess_bwd(const gs_frame* frame, const gs_prim_grads* grads, gs_stream stream);

/* The halves that gabsplat_render_bwd itself runs.  gabsplat_render_bwd_2d_zero does what
 * gabsplat_render_bwd_2d does and, inside the same kernel, zero-fills every array of grads (the
 * compositing walk is bound by instruction issue, the fill by HBM writes, so the fill costs little
 * time).  gabsplat_preprocess_bwd_prezeroed then writes only the rows of primitives that reach a
 * tile: the other rows must already be zero, i.e. grads must be the arrays just given to
 * gabsplat_render_bwd_2d_zero for this frame.  grads is required (GS_ERR_INVALID_ARG if NULL). */
gs_status gabsplat_render_bwd_2d_zero(const gs_frame* frame, const float* dL_drgb, const gs_prim_grads* grads,
                                      gs_stream stream);
gs_status gabsplat_preprocess_bwd_prezeroed(const gs_frame* frame, const gs_prim_grads* grads, gs_stream stream);

/* Photometric loss of Sec. 3.4.1 (its L1 part; L2 for gradient checks): mean over `count` values
 * of |image - target| or (image - target)^2.  Writes the loss (float64, device, 1 value) and
 * dL/d(image) (device, `count` floats).  scratch: device buffer of at least
 * gabsplat_loss_scratch_bytes(count) bytes. */
size_t gabsplat_loss_scratch_bytes(long long count);
gs_status gabsplat_loss(const float* image, const float* target, long long count, int kind, double* loss_out,
                        float* dL_dimage, void* scratch, gs_stream stream);

/* The loss above without a scratch argument, for callers that cannot allocate device memory:
 * e.g. a plug-in running inside another engine's frame loop whose allocator owns the device heap,
 * or a service under a fixed memory budget that allows no allocation once running.  The paper has
 * no counterpart; this is a packaging variant of gabsplat_loss with the same results (the loss
 * may differ in the last bits because the per-block sums are grouped differently).
 *  - The per-block partial sums live in a fixed 64 KB array inside the library (one double per
 *    4096 values), held by every GPU that loads the library until the process exits.
 *  - count must be at most GS_LOSS_NOALLOC_MAX_COUNT (33,554,432 values, e.g. a 3 x 3840 x 2160
 *    image fits); larger counts return GS_ERR_INVALID_ARG without launching anything.
 *  - The first call on each device looks up the array's device address (with that device
 *    current) and keeps it for the rest of the process; make that first call before any stream
 *    capture.  A cudaDeviceReset of a device invalidates the kept address: do not call this entry
 *    point on a device after resetting it.
 *  - All calls share the one array and each call overwrites the slots it reads, so nothing has to
 *    be cleared between calls, but calls that overlap on the GPU (different streams, or different
 *    host threads without ordering) race on it.  Issue them in order on one stream.
 *  - It never calls cudaMalloc, cudaFree or any allocating routine. */
#define GS_LOSS_NOALLOC_MAX_COUNT 33554432LL
gs_status gabsplat_loss_noalloc(const float* image, const float* target, long long count, int kind, double* loss_out,
                                float* dL_dimage, gs_stream stream);

/* Training objective of Sec. 3.4.1 (Eq. 11): L = (1 - lambda) L1 + lambda D-SSIM, the paper's
 * lambda being 0.2.  D-SSIM is 1 - mean SSIM, with SSIM the structural similarity index (Wang et
 * al. 2004, the metric of the paper's Sec. 4) computed per channel from window-weighted local
 * moments: an 11 x 11 Gaussian window of standard deviation 1.5 normalised to unit sum, zeros
 * outside the image, C1 = 0.01^2 and C2 = 0.03^2 (intensities in [0, 1]).  Both means run over all
 * channels x height x width values.
 *   image, target: [channels][height][width] float32, device; dL_dimage: the same shape, written
 *   with dL/dimage (the derivative of |d| is taken as 0 at d = 0); loss_out: one float64, device;
 *   scratch: device memory of gabsplat_loss_l1_dssim_scratch_bytes(channels, height, width) bytes.
 * The caller owns every buffer.  One fused kernel computes the loss and its gradient (float32
 * arithmetic, float64 for the final sums) plus a one-block reduction; both run on `stream`.
 * Returns GS_ERR_INVALID_ARG for a null pointer, channels outside [1, 64], a height or width
 * outside [1, 32768], or lambda outside [0, 1]. */
size_t gabsplat_loss_l1_dssim_scratch_bytes(int channels, int height, int width);
gs_status gabsplat_loss_l1_dssim(const float* image, const float* target, int channels, int height, int width,
                                 float lambda, double* loss_out, float* dL_dimage, void* scratch, gs_stream stream);

/* ---------------------------------------------------------------------------------------------
 * Frequency-adaptive density control (Sec. 3.4.2 and supplement B), on top of the adaptive density
 * control of 3DGS that the paper keeps: primitives whose mean screen-space positional gradient
 * reaches a threshold are cloned (small ones) or split into two (large ones), low-opacity and
 * (optionally) over-large ones are pruned, and every new primitive starts with its frequencies
 * and weights reset to small values, so it does not inherit its parent's high frequencies.
 * ------------------------------------------------------------------------------------------- */
typedef struct {
  float grad_threshold; /* mean |dL/dmu2D| (pixels) over the views that saw a primitive, at or
                           above which it is densified */
  float dense_scale;    /* largest scale up to which a candidate is cloned; larger ones are split */
  float min_opacity;    /* primitives with opacity below are pruned (the paper: 0.01) */
  float max_scale;      /* primitives whose largest scale exceeds it are pruned; <= 0: no such rule */
  float split_divisor;  /* scales of split children = parent's / split_divisor (3DGS: 0.8 x 2 = 1.6) */
  float child_freq;     /* every frequency coordinate of a new primitive (the paper: 0.001) */
  float child_weight;   /* every weight of a new primitive (the paper: 0.01) */
} gs_densify_config;

/* Writable attribute arrays, laid out as in gs_prims (sh/freqs/weights in the storage type). */
typedef struct {
  float* means;
  float* scales;
  float* quats;
  float* opacity;
  void* sh;
  void* freqs;
  void* weights;
} gs_prim_arrays;

/* One training view's statistics, after gabsplat_preprocess_bwd: every primitive that reached at
 * least one tile of the frame's view adds sqrt(gx^2 + gy^2) of its means2d gradient (pixels,
 * [n][2] float32, the gs_prim_grads.means2d output) to grad_accum[i] and 1 to denom[i] ([n]
 * float32, device, caller-owned; start them at zero and zero them after gabsplat_densify).
 * Single correctly rounded float32 operations. */
gs_status gabsplat_densify_accumulate(const gs_frame* frame, const float* means2d_grad, float* grad_accum,
                                      float* denom, gs_stream stream);

/* Clone / split / prune in one compaction.  Per primitive i, in float32:
 *   g = grad_accum[i] / denom[i] (0 if denom is 0); candidate if g >= grad_threshold;
 *   s_max = largest scale; candidates with s_max <= dense_scale are cloned, the others split;
 *   pruned: opacity < min_opacity, or max_scale > 0 and s_max > max_scale (split children are
 *   tested with their own scales).
 * Output rows (out, capacity out_capacity >= 2 n rows), in this order: the kept originals, the
 * clones, then two children per split, each segment in index order.  Clones and children copy
 * rotation, opacity and SH; their frequencies are child_freq and weights child_weight.  Child c
 * of primitive i sits at mu + R(q) (s * z) with z = split_noise[i][c][0..2] (float32 [n][2][3],
 * standard normal samples drawn by the caller) and has scale s / split_divisor.
 * counts (device, 4 ints): {rows written, originals, clones, split children}; the count never
 * leaves the device.  n <= 2^30 - 1.  scratch: gabsplat_densify_scratch_bytes(n) bytes of device
 * memory.  Input and output arrays must not overlap; out->quats 16-byte aligned. */
size_t gabsplat_densify_scratch_bytes(int n);
gs_status gabsplat_densify(const gs_prims* in, const float* grad_accum, const float* denom, const float* split_noise,
                           const gs_densify_config* cfg, const gs_prim_arrays* out, long long out_capacity,
                           int* counts, void* scratch, gs_stream stream);

/* The periodic reset (the paper: every 3000 iterations, with the opacity reset): opacity =
 * min(opacity, opacity_cap) and every weight = weight, in place on n primitives with K
 * components stored as `storage`. */
gs_status gabsplat_reset_opacity_weights(const gs_prim_arrays* prims, int n, int K, int storage, float opacity_cap,
                                         float weight, gs_stream stream);

/* ---------------------------------------------------------------------------------------------
 * Batched frames (serving).  A batch renders up to GS_MAX_VIEWS views -- each a camera with its own
 * resolution over one resident scene -- with one launch sequence (forward only): the views'
 * primitives, tiles and pixels are concatenated, so one sort and one persistent compositing launch
 * serve all of them, and every view's image is bit-identical to rendering that view alone with
 * gabsplat_preprocess / gabsplat_bin_sort / gabsplat_render_fwd.  All views of a batch share K,
 * sh_degree and storage (those of the batch frame) and the gs_config.
 * ------------------------------------------------------------------------------------------- */
typedef struct {
  gs_prims prims;   /* device arrays of the view's scene */
  gs_camera cam;    /* the view's camera and resolution */
  float* out_rgb;   /* device [3][cam.height][cam.width], required */
  float* out_T;     /* device [cam.height][cam.width], may be NULL */
} gs_view;

/* Capacity of a batched workspace: at most max_views views whose primitive counts sum to at most
 * max_prims, tile counts to max_tiles and pixel counts to max_pixels, with at most pair_capacity
 * (tile, primitive) pairs in total. */
typedef struct {
  int max_views, K, sh_degree, storage;
  unsigned long long max_prims, max_tiles, max_pixels, pair_capacity;
  void* ws;          /* device, 256-byte aligned, zero-filled once (gabsplat_batch_workspace_init) */
  size_t ws_bytes;
} gs_batch_frame;

size_t gabsplat_batch_workspace_size(int max_views, int K, int sh_degree, unsigned long long max_prims,
                                     unsigned long long max_tiles, unsigned long long max_pixels,
                                     unsigned long long pair_capacity);
gs_status gabsplat_batch_workspace_init(const gs_batch_frame* frame, gs_stream stream);

/* Render `nviews` views (Sec. 3.3, Eq. 9-10 per view) with direct launches on `stream`.
 * GS_ERR_CAPACITY (host, nothing launched) if the views exceed the frame's primitive, tile or
 * pixel capacity; pair overflow is reported on the device as for single frames. */
gs_status gabsplat_render_batch(const gs_batch_frame* frame, const gs_view* views, int nviews, const gs_config* cfg,
                                gs_stream stream);

/* Asynchronously copies the 16-byte status record {int status; unsigned epoch; unsigned long long pairs}
 * of the batch's workspace to `dst` (pinned host or device memory) on `stream`. */
gs_status gabsplat_batch_status_copy(const gs_batch_frame* frame, void* dst, gs_stream stream);

/* A CUDA graph of the batch launch sequence, captured once per workspace on `stream` (which must
 * not be the legacy default stream) and replayed per batch: each launch writes the new view table
 * into the graph's first kernel node, so replays need no re-capture.  The graph executor is host
 * memory allocated by the library (malloc); destroy it with gabsplat_batch_graph_destroy.  Launches
 * of one graph must not overlap on the device (they share the workspace). */
typedef struct gs_batch_graph gs_batch_graph;
gs_status gabsplat_batch_graph_create(const gs_batch_frame* frame, const gs_config* cfg, gs_stream stream,
                                      gs_batch_graph** out);
gs_status gabsplat_batch_graph_launch(gs_batch_graph* graph, const gs_view* views, int nviews, gs_stream stream);
void gabsplat_batch_graph_destroy(gs_batch_graph* graph);

/* Synchronises `stream`, then reads the workspace status word.  *status = device-side
 * gs_status of the last frame, *pairs = number of (tile, primitive) pairs it produced (the
 * required capacity when *status == GS_ERR_CAPACITY).  Either output pointer may be NULL. */
gs_status gabsplat_device_status(const gs_frame* frame, int* status, unsigned long long* pairs, gs_stream stream);

/* Device pointers into the workspace of `frame`.  Reads the workspace header with a synchronous
 * copy (the sorted pairs end in one of two buffers, decided on the device). */
gs_status gabsplat_workspace_views(const gs_frame* frame, gs_ws_views* out);

/* Human-readable name of a status code (static string). */
const char* gabsplat_status_string(gs_status s);

/* Library version string. */
const char* gabsplat_version(void);

#ifdef __cplusplus
}
#endif
#endif /* GABSPLAT_H */
