// C ABI of the rasterizer: argument checks, workspace layout and stage launches.
#include <cmath>
#include <cstring>

#include "common.cuh"

namespace gs {

static inline size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

WsLayout make_layout(u32 n_prims, int K, u32 n_tiles, u64 n_pixels, u64 capacity) {
  WsLayout L;
  memset(&L, 0, sizeof(L));
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t o = off;
    off = al256(off + (bytes ? bytes : 1));
    return o;
  };
  L.n_prims = n_prims;
  L.n_tiles = n_tiles;
  L.n_pixels = n_pixels;
  L.capacity = capacity;
  L.K = K;
  L.rec_f = rec_floats(K);
  L.g2d_f = g2d_floats(K);
  L.n_chunks = (n_prims + CHUNK - 1) / CHUNK;
  const u64 sort_items = capacity > n_prims ? capacity : n_prims;   // pairs, or active primitives
  L.n_parts = (u32)((sort_items + SORT_TILE - 1) / SORT_TILE);          // partitions of either sort, at most
  L.header = take(sizeof(WsHeader));
  L.table = take(sizeof(FrameTable));
  L.records = take((size_t)n_prims * L.rec_f * sizeof(float));
  L.touched = take((size_t)n_prims * 4);
  L.offsets = take((size_t)n_prims * 4);
  L.order = take((size_t)n_prims * 4);
  L.active = take((size_t)n_prims * 4);
  L.rank_of = take((size_t)n_prims * 4);
  L.dkeys0 = take((size_t)n_prims * 8);
  L.dkeys1 = take((size_t)n_prims * 8);
  L.scan_partials = take((size_t)(L.n_chunks ? L.n_chunks : 1) * 8);
  L.rank_partials = take((size_t)(L.n_chunks ? L.n_chunks : 1) * 8);
  L.keys0 = take((size_t)capacity * 8);
  L.keys1 = take((size_t)capacity * 8);
  L.hist = take((size_t)MAX_PASSES * RADIX * 4);
  L.sort_status = take((size_t)(L.n_parts ? L.n_parts : 1) * RADIX * 8);
  L.ranges = take((size_t)n_tiles * 8);
  L.tile_order = take((size_t)n_tiles * 4);
  L.cmask = take((size_t)CMASK_PLANES * (capacity / 32 + n_tiles + 2) * 4);
  L.T_final = take((size_t)n_pixels * 4);
  L.n_contrib = take((size_t)n_pixels * 4);
  L.n_eval = take((size_t)n_pixels * 4);
  L.n_reach = take((size_t)n_pixels * 4);
  L.n_comp = take((size_t)n_pixels * 4);
  L.grad2d = take((size_t)n_prims * L.g2d_f * sizeof(float));
  L.total = off;
  return L;
}

WsPtrs make_ptrs(const WsLayout& L, void* ws) {
  char* b = reinterpret_cast<char*>(ws);
  WsPtrs p;
  p.hdr = reinterpret_cast<WsHeader*>(b + L.header);
  p.tbl = reinterpret_cast<const FrameTable*>(b + L.table);
  p.records = reinterpret_cast<float*>(b + L.records);
  p.touched = reinterpret_cast<u32*>(b + L.touched);
  p.offsets = reinterpret_cast<u32*>(b + L.offsets);
  p.order = reinterpret_cast<u32*>(b + L.order);
  p.active = reinterpret_cast<u32*>(b + L.active);
  p.rank_of = reinterpret_cast<u32*>(b + L.rank_of);
  p.dkeys0 = reinterpret_cast<u64*>(b + L.dkeys0);
  p.dkeys1 = reinterpret_cast<u64*>(b + L.dkeys1);
  p.scan_partials = reinterpret_cast<u64*>(b + L.scan_partials);
  p.rank_partials = reinterpret_cast<u64*>(b + L.rank_partials);
  p.keys0 = reinterpret_cast<u64*>(b + L.keys0);
  p.keys1 = reinterpret_cast<u64*>(b + L.keys1);
  p.hist = reinterpret_cast<u32*>(b + L.hist);
  p.sort_status = reinterpret_cast<u64*>(b + L.sort_status);
  p.ranges = reinterpret_cast<uint2*>(b + L.ranges);
  p.tile_order = reinterpret_cast<u32*>(b + L.tile_order);
  p.cmask = reinterpret_cast<u32*>(b + L.cmask);
  p.cmask_plane = (u32)(L.capacity / 32 + L.n_tiles + 2);
  p.T_final = reinterpret_cast<float*>(b + L.T_final);
  p.n_contrib = reinterpret_cast<u32*>(b + L.n_contrib);
  p.n_eval = reinterpret_cast<u32*>(b + L.n_eval);
  p.n_reach = reinterpret_cast<u32*>(b + L.n_reach);
  p.n_comp = reinterpret_cast<u32*>(b + L.n_comp);
  p.grad2d = reinterpret_cast<float*>(b + L.grad2d);
  p.capacity = L.capacity;
  p.n_chunks = L.n_chunks;
  p.n_parts = L.n_parts;
  return p;
}

static int g_sms = 0;
static Launch make_launch(gs_stream s) {
  if (!g_sms) g_sms = device_sm_count();
  Launch L;
  L.sm_count = g_sms;
  L.stream = reinterpret_cast<cudaStream_t>(s);
  return L;
}

int tile_bits(u32 ntiles) {
  int b = 0;
  while (b < 32 && ((u64)1 << b) < (u64)ntiles) ++b;
  return b;
}
int tile_passes(u32 ntiles) { return (tile_bits(ntiles) + RADIX_BITS - 1) / RADIX_BITS; }

// Depth keys of culled-in primitives lie in (bits(znear), bits(zfar)]: positive floats order like their
// bit patterns, so subtracting bits(znear) leaves a value below 2^depth_bits, and the depth sort needs
// ceil(depth_bits / 8) digit passes.  The tile sort needs ceil(tile bits / 8) (none for one tile).
void set_depth_window(FrameTable& t, float znear_min, float zfar_max) {
  u32 lo, hi;
  memcpy(&lo, &znear_min, 4);
  memcpy(&hi, &zfar_max, 4);
  int db = 1;
  while (db < 32 && ((u64)(hi - lo) >> db) != 0) ++db;
  t.depth_base = lo;
  t.depth_bits = db;
  t.dpasses_needed = (db + RADIX_BITS - 1) / RADIX_BITS;
  if (t.dpasses_needed > DPASSES) t.dpasses_needed = DPASSES;
  t.tpasses_needed = tile_passes(t.total_tiles);
  if (t.tpasses_needed > t.tpasses) t.tpasses_needed = t.tpasses;
}

static bool frame_sizes_ok(int n, int K, int sh_degree, int width, int height, u64 cap) {
  return n >= 0 && K >= 0 && K <= GS_MAX_K && sh_degree >= 0 && sh_degree <= GS_MAX_SH_DEGREE && width > 0 &&
         height > 0 && width <= 32768 && height <= 32768 && cap < (1ull << 32);
}

// Host-side description of a single-view frame, enough for every launcher.
static gs_status frame_meta(const gs_frame* f, FrameTable& t, WsLayout& L) {
  if (!f || !f->ws) return GS_ERR_INVALID_ARG;
  if (!frame_sizes_ok(f->n, f->K, f->sh_degree, f->width, f->height, f->pair_capacity)) return GS_ERR_INVALID_ARG;
  if (f->storage != GS_F32 && f->storage != GS_BF16) return GS_ERR_INVALID_ARG;
  if (reinterpret_cast<uintptr_t>(f->ws) & 255) return GS_ERR_WORKSPACE;
  memset(&t, 0, sizeof(t));
  t.storage = f->storage;   // every stage dispatches on the frame's storage type
  const int tx = (f->width + TILE - 1) / TILE, ty = (f->height + TILE - 1) / TILE;
  t.nviews = 1;
  t.K = f->K;
  t.sh_degree = f->sh_degree;
  t.total_prims = (u32)f->n;
  t.total_tiles = (u32)(tx * ty);
  t.total_pixels = (u64)f->width * f->height;
  t.tpasses = tile_passes(t.total_tiles);
  t.launch_prims = t.total_prims;
  t.launch_tiles = t.total_tiles;
  t.v[0].n = f->n;
  t.v[0].width = f->width;
  t.v[0].height = f->height;
  t.v[0].tiles_x = tx;
  t.v[0].tiles_y = ty;
  L = make_layout(t.total_prims, f->K, t.total_tiles, t.total_pixels, f->pair_capacity);
  if (f->ws_bytes < L.total) return GS_ERR_WORKSPACE;
  return GS_OK;
}

static gs_status from_cuda(cudaError_t e) { return e == cudaSuccess ? GS_OK : GS_ERR_CUDA; }

}  // namespace gs

using namespace gs;

extern "C" {

size_t gabsplat_workspace_size(int n, int K, int sh_degree, int width, int height, unsigned long long pair_capacity) {
  if (!frame_sizes_ok(n, K, sh_degree, width, height, pair_capacity)) return 0;
  const u32 tiles = (u32)(((width + TILE - 1) / TILE) * ((height + TILE - 1) / TILE));
  return make_layout((u32)n, K, tiles, (u64)width * height, pair_capacity).total;
}

gs_status gabsplat_workspace_init(const gs_frame* frame, gs_stream stream) {
  FrameTable t;
  WsLayout L;
  const gs_status s = frame_meta(frame, t, L);
  if (s != GS_OK) return s;
  return from_cuda(cudaMemsetAsync(frame->ws, 0, L.total, reinterpret_cast<cudaStream_t>(stream)));
}

gs_status gabsplat_preprocess(const gs_frame* frame, const gs_prims* pr, const gs_camera* cam, const gs_config* cfg,
                              gs_stream stream) {
  FrameTable t;
  WsLayout L;
  gs_status s = frame_meta(frame, t, L);
  if (s != GS_OK) return s;
  if (!pr || !cam || !cfg) return GS_ERR_INVALID_ARG;
  if (pr->n != frame->n || pr->K != frame->K || pr->sh_degree != frame->sh_degree) return GS_ERR_INVALID_ARG;
  if (pr->storage != frame->storage) return GS_ERR_INVALID_ARG;
  if (cam->width != frame->width || cam->height != frame->height) return GS_ERR_INVALID_ARG;
  if (pr->n > 0 && (!pr->means || !pr->scales || !pr->quats || !pr->opacity || !pr->sh)) return GS_ERR_INVALID_ARG;
  if (pr->n > 0 && pr->K > 0 && (!pr->freqs || !pr->weights)) return GS_ERR_INVALID_ARG;
  if (reinterpret_cast<uintptr_t>(pr->quats) & 15) return GS_ERR_INVALID_ARG;
  if (!(cam->fx > 0.f) || !(cam->fy > 0.f) || !(cam->znear > 0.f) || !(cam->zfar > cam->znear))
    return GS_ERR_INVALID_ARG;
  if ((cfg->flags & ~(unsigned)GS_FLAG_Z_ATTENUATION) != 0 || !(cfg->eps2d >= 0.f) || !(cfg->alpha_max > 0.f) || !(cfg->alpha_max < 1.f) ||
      !(cfg->alpha_min > 0.f) || !(cfg->T_min > 0.f))
    return GS_ERR_INVALID_ARG;
  t.storage = pr->storage;
  t.eps2d = cfg->eps2d;
  t.alpha_max = cfg->alpha_max;
  t.alpha_min = cfg->alpha_min;
  t.T_min = cfg->T_min;
  t.flags = cfg->flags;
  for (int i = 0; i < 3; ++i) t.bg[i] = cfg->bg[i];
  ViewDesc& V = t.v[0];
  V.means = pr->means;
  V.scales = pr->scales;
  V.quats = pr->quats;
  V.opacity = pr->opacity;
  V.sh = pr->sh;
  V.freqs = pr->freqs;
  V.weights = pr->weights;
  V.sh_degree = pr->sh_degree;
  for (int i = 0; i < 9; ++i) V.R[i] = cam->R[i];
  for (int i = 0; i < 3; ++i) V.t[i] = cam->t[i];
  V.fx = cam->fx; V.fy = cam->fy; V.cx = cam->cx; V.cy = cam->cy;
  V.znear = cam->znear; V.zfar = cam->zfar;
  for (int i = 0; i < 3; ++i)   // camera centre -R^T t
    V.campos[i] = -(cam->R[i] * cam->t[0] + cam->R[3 + i] * cam->t[1] + cam->R[6 + i] * cam->t[2]);
  set_depth_window(t, cam->znear, cam->zfar);
  const WsPtrs p = make_ptrs(L, frame->ws);
  const Launch lc = make_launch(stream);
  cudaError_t e = launch_setup(t, p, lc);
  if (e == cudaSuccess) e = launch_preprocess(t, p, lc);
  return from_cuda(e);
}

gs_status gabsplat_bin_sort(const gs_frame* frame, gs_stream stream) {
  FrameTable t;
  WsLayout L;
  const gs_status s = frame_meta(frame, t, L);
  if (s != GS_OK) return s;
  return from_cuda(launch_bin_sort(t, make_ptrs(L, frame->ws), make_launch(stream)));
}

gs_status gabsplat_render_fwd(const gs_frame* frame, float* out_rgb, float* out_T, gs_stream stream) {
  FrameTable t;
  WsLayout L;
  const gs_status s = frame_meta(frame, t, L);
  if (s != GS_OK) return s;
  if (!out_rgb) return GS_ERR_INVALID_ARG;
  return from_cuda(launch_render_fwd(t, make_ptrs(L, frame->ws), out_rgb, out_T, make_launch(stream), true));
}

gs_status gabsplat_render_fwd_stats(const gs_frame* frame, float* out_rgb, float* out_T, gs_stream stream) {
  FrameTable t;
  WsLayout L;
  const gs_status s = frame_meta(frame, t, L);
  if (s != GS_OK) return s;
  if (!out_rgb) return GS_ERR_INVALID_ARG;
  return from_cuda(launch_render_fwd(t, make_ptrs(L, frame->ws), out_rgb, out_T, make_launch(stream), true, true));
}

gs_status gabsplat_render_fwd_only(const gs_frame* frame, float* out_rgb, float* out_T, gs_stream stream) {
  FrameTable t;
  WsLayout L;
  const gs_status s = frame_meta(frame, t, L);
  if (s != GS_OK) return s;
  if (!out_rgb) return GS_ERR_INVALID_ARG;
  return from_cuda(launch_render_fwd(t, make_ptrs(L, frame->ws), out_rgb, out_T, make_launch(stream), false));
}

gs_status gabsplat_render_freq_map(const gs_frame* frame, float* out_map, gs_stream stream) {
  FrameTable t;
  WsLayout L;
  const gs_status s = frame_meta(frame, t, L);
  if (s != GS_OK) return s;
  if (!out_map) return GS_ERR_INVALID_ARG;
  return from_cuda(launch_render_freq_map(t, make_ptrs(L, frame->ws), out_map, make_launch(stream)));
}

// The 2D adjoint (grad2d rows cleared first); with grads, the kernel also zero-fills them.
static gs_status render_bwd_2d(const gs_frame* frame, const float* dL_drgb, const gs_prim_grads* grads,
                               gs_stream stream) {
  FrameTable t;
  WsLayout L;
  const gs_status s = frame_meta(frame, t, L);
  if (s != GS_OK) return s;
  if (!dL_drgb) return GS_ERR_INVALID_ARG;
  const WsPtrs p = make_ptrs(L, frame->ws);
  if (!grads) return from_cuda(launch_render_bwd(t, p, dL_drgb, nullptr, make_launch(stream)));
  const ZeroJob z = make_zero_job(*grads, t.v[0].n, t.K, (t.sh_degree + 1) * (t.sh_degree + 1), t.total_tiles);
  return from_cuda(launch_render_bwd(t, p, dL_drgb, &z, make_launch(stream)));
}

static gs_status preprocess_bwd(const gs_frame* frame, const gs_prim_grads* grads, bool prezeroed,
                                gs_stream stream) {
  FrameTable t;
  WsLayout L;
  const gs_status s = frame_meta(frame, t, L);
  if (s != GS_OK) return s;
  if (!grads) return GS_ERR_INVALID_ARG;
  return from_cuda(launch_preprocess_bwd(t, make_ptrs(L, frame->ws), *grads, prezeroed, make_launch(stream)));
}

gs_status gabsplat_render_bwd_2d(const gs_frame* frame, const float* dL_drgb, gs_stream stream) {
  return render_bwd_2d(frame, dL_drgb, nullptr, stream);
}

gs_status gabsplat_preprocess_bwd(const gs_frame* frame, const gs_prim_grads* grads, gs_stream stream) {
  return preprocess_bwd(frame, grads, false, stream);
}

gs_status gabsplat_render_bwd_2d_zero(const gs_frame* frame, const float* dL_drgb, const gs_prim_grads* grads,
                                      gs_stream stream) {
  if (!grads) return GS_ERR_INVALID_ARG;
  return render_bwd_2d(frame, dL_drgb, grads, stream);
}

gs_status gabsplat_preprocess_bwd_prezeroed(const gs_frame* frame, const gs_prim_grads* grads, gs_stream stream) {
  return preprocess_bwd(frame, grads, true, stream);
}

gs_status gabsplat_render_bwd(const gs_frame* frame, const float* dL_drgb, const gs_prim_grads* grads,
                              gs_stream stream) {
  const gs_status s = gabsplat_render_bwd_2d_zero(frame, dL_drgb, grads, stream);
  if (s != GS_OK) return s;
  return gabsplat_preprocess_bwd_prezeroed(frame, grads, stream);
}

size_t gabsplat_loss_scratch_bytes(long long count) {
  (void)count;
  return (size_t)1024 * sizeof(double);
}

gs_status gabsplat_loss(const float* image, const float* target, long long count, int kind, double* loss_out,
                        float* dL_dimage, void* scratch, gs_stream stream) {
  if (!image || !target || !loss_out || !dL_dimage || !scratch || count <= 0) return GS_ERR_INVALID_ARG;
  if (kind != GS_LOSS_L1 && kind != GS_LOSS_L2) return GS_ERR_INVALID_ARG;
  if (!g_sms) g_sms = device_sm_count();
  int blocks = g_sms * 4;
  if (blocks > 1024) blocks = 1024;
  return from_cuda(launch_loss(image, target, count, kind, loss_out, dL_dimage, reinterpret_cast<double*>(scratch),
                               blocks, reinterpret_cast<cudaStream_t>(stream)));
}

static bool l1_dssim_sizes_ok(int channels, int height, int width) {
  return channels >= 1 && channels <= 64 && height >= 1 && width >= 1 && height <= 32768 && width <= 32768;
}

size_t gabsplat_loss_l1_dssim_scratch_bytes(int channels, int height, int width) {
  if (!l1_dssim_sizes_ok(channels, height, width)) return 0;
  return l1_dssim_partials(channels, height, width) * sizeof(double);
}

gs_status gabsplat_loss_l1_dssim(const float* image, const float* target, int channels, int height, int width,
                                 float lambda, double* loss_out, float* dL_dimage, void* scratch, gs_stream stream) {
  if (!image || !target || !loss_out || !dL_dimage || !scratch) return GS_ERR_INVALID_ARG;
  if (!l1_dssim_sizes_ok(channels, height, width)) return GS_ERR_INVALID_ARG;
  if (!(lambda >= 0.f && lambda <= 1.f)) return GS_ERR_INVALID_ARG;
  return from_cuda(launch_l1_dssim(image, target, channels, height, width, lambda, loss_out, dL_dimage,
                                   reinterpret_cast<double*>(scratch), reinterpret_cast<cudaStream_t>(stream)));
}

gs_status gabsplat_densify_accumulate(const gs_frame* frame, const float* means2d_grad, float* grad_accum,
                                      float* denom, gs_stream stream) {
  FrameTable t;
  WsLayout L;
  const gs_status s = frame_meta(frame, t, L);
  if (s != GS_OK) return s;
  if (frame->n > 0 && (!means2d_grad || !grad_accum || !denom)) return GS_ERR_INVALID_ARG;
  if (!g_sms) g_sms = device_sm_count();
  const WsPtrs p = make_ptrs(L, frame->ws);
  return from_cuda(launch_densify_accumulate(p.touched, frame->n, means2d_grad, grad_accum, denom, g_sms,
                                             reinterpret_cast<cudaStream_t>(stream)));
}

gs_status gabsplat_device_status(const gs_frame* frame, int* status, unsigned long long* pairs, gs_stream stream) {
  FrameTable t;
  WsLayout L;
  const gs_status s = frame_meta(frame, t, L);
  if (s != GS_OK) return s;
  WsHeader h;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  cudaError_t e =
      cudaMemcpyAsync(&h, reinterpret_cast<char*>(frame->ws) + L.header, sizeof(h), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return GS_ERR_CUDA;
  if (status) *status = h.status;
  if (pairs) *pairs = h.pairs;
  return GS_OK;
}

gs_status gabsplat_workspace_views(const gs_frame* frame, gs_ws_views* out) {
  FrameTable t;
  WsLayout L;
  const gs_status s = frame_meta(frame, t, L);
  if (s != GS_OK) return s;
  if (!out) return GS_ERR_INVALID_ARG;
  const WsPtrs p = make_ptrs(L, frame->ws);
  WsHeader h;
  if (cudaMemcpy(&h, p.hdr, sizeof(h), cudaMemcpyDeviceToHost) != cudaSuccess) return GS_ERR_CUDA;
  const bool odd = h.sorted_buf != 0;
  out->records = p.records;
  out->touched = p.touched;
  out->offsets = p.offsets;
  out->order = p.order;
  out->n_active = h.n_active;
  out->keys_sorted = odd ? p.keys1 : p.keys0;
  out->keys_unsorted = p.keys0;     // valid between gabsplat_preprocess and gabsplat_bin_sort
  out->ranges = reinterpret_cast<unsigned*>(p.ranges);
  out->T_final = p.T_final;
  out->n_contrib = p.n_contrib;
  out->n_eval = p.n_eval;
  out->n_reach = p.n_reach;
  out->n_comp = p.n_comp;
  out->grad2d = p.grad2d;
  out->record_floats = L.rec_f;
  out->grad2d_floats = L.g2d_f;
  out->tiles_x = t.v[0].tiles_x;
  out->tiles_y = t.v[0].tiles_y;
  return GS_OK;
}

const char* gabsplat_status_string(gs_status s) {
  switch (s) {
    case GS_OK: return "ok";
    case GS_ERR_INVALID_ARG: return "invalid argument";
    case GS_ERR_CAPACITY: return "pair capacity exceeded";
    case GS_ERR_TIMEOUT: return "device wait timed out";
    case GS_ERR_CUDA: return "CUDA error";
    case GS_ERR_NONFINITE: return "non-finite projected value";
    case GS_ERR_WORKSPACE: return "workspace too small or misaligned";
    default: return "unknown status";
  }
}

const char* gabsplat_version(void) { return "gabsplat 0.1 sm_103a"; }

}  // extern "C"
