// Batched frames for serving: up to GS_MAX_VIEWS views (each a camera over one resident scene, with
// its own resolution) rendered by one launch sequence.  Views are concatenated: primitive records,
// tiles and pixels of view v start at its prim/tile/pixel base, tile ids in the sort keys are
// global, so one sort and one persistent compositing launch serve every view and each view's
// result is bit-identical to rendering it alone.  A CUDA-graph executor captures the sequence
// once per workspace and replays it with a new view table.
#include <cstdlib>
#include <cstring>

#include "common.cuh"

namespace gs {
const void* setup_kernel_fn();
}

using namespace gs;

struct gs_batch_graph {
  cudaGraph_t graph;
  cudaGraphExec_t exec;
  cudaGraphNode_t setup_node;
  cudaKernelNodeParams setup_params;
  gs_batch_frame frame;
  gs_config cfg;
  WsPtrs ptrs;
};

namespace {

bool batch_sizes_ok(const gs_batch_frame* f) {
  return f && f->ws && f->max_views >= 1 && f->max_views <= GS_MAX_VIEWS && f->K >= 0 && f->K <= GS_MAX_K &&
         f->sh_degree >= 0 && f->sh_degree <= GS_MAX_SH_DEGREE && (f->storage == GS_F32 || f->storage == GS_BF16) &&
         f->max_prims < (1ull << 31) && f->max_tiles >= 1 && f->max_tiles < (1ull << 31) && f->max_pixels >= 1 &&
         f->pair_capacity < (1ull << 32);
}

WsLayout batch_layout(const gs_batch_frame* f) {
  return make_layout((u32)f->max_prims, f->K, (u32)f->max_tiles, f->max_pixels, f->pair_capacity);
}

// Host-side frame table for a list of views.  Returns GS_OK or the reason it does not fit.
gs_status build_batch_table(const gs_batch_frame* f, const gs_view* views, int nviews, const gs_config* cfg,
                            FrameTable& t) {
  if (nviews < 0 || nviews > f->max_views || (nviews > 0 && !views) || !cfg) return GS_ERR_INVALID_ARG;
  if ((cfg->flags & ~(unsigned)GS_FLAG_Z_ATTENUATION) != 0 || !(cfg->eps2d >= 0.f) || !(cfg->alpha_max > 0.f) || !(cfg->alpha_max < 1.f) ||
      !(cfg->alpha_min > 0.f) || !(cfg->T_min > 0.f))
    return GS_ERR_INVALID_ARG;
  memset(&t, 0, sizeof(t));
  t.nviews = nviews;
  t.K = f->K;
  t.storage = f->storage;
  t.sh_degree = f->sh_degree;
  t.eps2d = cfg->eps2d;
  t.alpha_max = cfg->alpha_max;
  t.alpha_min = cfg->alpha_min;
  t.T_min = cfg->T_min;
  t.flags = cfg->flags;
  for (int i = 0; i < 3; ++i) t.bg[i] = cfg->bg[i];
  t.tpasses = tile_passes((u32)f->max_tiles);   // fixed per workspace, so graph replays agree
  t.launch_prims = (u32)f->max_prims;
  t.launch_tiles = (u32)f->max_tiles;
  u64 prims = 0, tiles = 0, pixels = 0;
  for (int v = 0; v < nviews; ++v) {
    const gs_prims& pr = views[v].prims;
    const gs_camera& cam = views[v].cam;
    if (pr.K != f->K || pr.sh_degree != f->sh_degree || pr.storage != f->storage || pr.n < 0) return GS_ERR_INVALID_ARG;
    if (pr.n > 0 && (!pr.means || !pr.scales || !pr.quats || !pr.opacity || !pr.sh)) return GS_ERR_INVALID_ARG;
    if (pr.n > 0 && pr.K > 0 && (!pr.freqs || !pr.weights)) return GS_ERR_INVALID_ARG;
    if (reinterpret_cast<uintptr_t>(pr.quats) & 15) return GS_ERR_INVALID_ARG;
    if (cam.width <= 0 || cam.height <= 0 || cam.width > 32768 || cam.height > 32768) return GS_ERR_INVALID_ARG;
    if (!(cam.fx > 0.f) || !(cam.fy > 0.f) || !(cam.znear > 0.f) || !(cam.zfar > cam.znear)) return GS_ERR_INVALID_ARG;
    if (!views[v].out_rgb) return GS_ERR_INVALID_ARG;
    ViewDesc& V = t.v[v];
    V.means = pr.means;
    V.scales = pr.scales;
    V.quats = pr.quats;
    V.opacity = pr.opacity;
    V.sh = pr.sh;
    V.freqs = pr.freqs;
    V.weights = pr.weights;
    V.out_rgb = views[v].out_rgb;
    V.out_T = views[v].out_T;
    V.dL_drgb = nullptr;
    V.n = pr.n;
    V.sh_degree = pr.sh_degree;
    for (int i = 0; i < 9; ++i) V.R[i] = cam.R[i];
    for (int i = 0; i < 3; ++i) V.t[i] = cam.t[i];
    V.fx = cam.fx; V.fy = cam.fy; V.cx = cam.cx; V.cy = cam.cy;
    V.znear = cam.znear; V.zfar = cam.zfar;
    for (int i = 0; i < 3; ++i)
      V.campos[i] = -(cam.R[i] * cam.t[0] + cam.R[3 + i] * cam.t[1] + cam.R[6 + i] * cam.t[2]);
    V.width = cam.width;
    V.height = cam.height;
    V.tiles_x = (cam.width + TILE - 1) / TILE;
    V.tiles_y = (cam.height + TILE - 1) / TILE;
    V.prim_base = (u32)prims;
    V.tile_base = (u32)tiles;
    V.pix_base = pixels;
    prims += (u64)pr.n;
    tiles += (u64)V.tiles_x * V.tiles_y;
    pixels += (u64)cam.width * cam.height;
  }
  if (prims > f->max_prims || tiles > f->max_tiles || pixels > f->max_pixels) return GS_ERR_CAPACITY;
  t.total_prims = (u32)prims;
  t.total_tiles = (u32)tiles;
  t.total_pixels = pixels;
  float zn = 3.0e38f, zf = 0.f;
  for (int v = 0; v < nviews; ++v) {
    zn = fminf(zn, views[v].cam.znear);
    zf = fmaxf(zf, views[v].cam.zfar);
  }
  if (nviews == 0) zn = zf = 1.f;
  set_depth_window(t, zn, zf);
  return GS_OK;
}

cudaError_t launch_sequence(const FrameTable& t, const WsPtrs& p, cudaStream_t s) {
  static int sms = 0;
  if (!sms) sms = device_sm_count();
  Launch L;
  L.sm_count = sms;
  L.stream = s;
  cudaError_t e = launch_setup(t, p, L);
  if (e == cudaSuccess) e = launch_preprocess(t, p, L);
  if (e == cudaSuccess) e = launch_bin_sort(t, p, L);
  if (e == cudaSuccess) e = launch_render_fwd(t, p, nullptr, nullptr, L, false);
  return e;
}

}  // namespace

extern "C" {

size_t gabsplat_batch_workspace_size(int max_views, int K, int sh_degree, unsigned long long max_prims,
                                     unsigned long long max_tiles, unsigned long long max_pixels,
                                     unsigned long long pair_capacity) {
  gs_batch_frame f;
  memset(&f, 0, sizeof(f));
  f.max_views = max_views;
  f.K = K;
  f.sh_degree = sh_degree;
  f.storage = GS_F32;
  f.max_prims = max_prims;
  f.max_tiles = max_tiles;
  f.max_pixels = max_pixels;
  f.pair_capacity = pair_capacity;
  f.ws = reinterpret_cast<void*>(256);
  if (!batch_sizes_ok(&f)) return 0;
  return batch_layout(&f).total;
}

gs_status gabsplat_batch_workspace_init(const gs_batch_frame* f, gs_stream stream) {
  if (!batch_sizes_ok(f)) return GS_ERR_INVALID_ARG;
  const WsLayout L = batch_layout(f);
  if (f->ws_bytes < L.total || (reinterpret_cast<uintptr_t>(f->ws) & 255)) return GS_ERR_WORKSPACE;
  return cudaMemsetAsync(f->ws, 0, L.total, reinterpret_cast<cudaStream_t>(stream)) == cudaSuccess ? GS_OK
                                                                                                     : GS_ERR_CUDA;
}

gs_status gabsplat_render_batch(const gs_batch_frame* f, const gs_view* views, int nviews, const gs_config* cfg,
                                gs_stream stream) {
  if (!batch_sizes_ok(f)) return GS_ERR_INVALID_ARG;
  const WsLayout L = batch_layout(f);
  if (f->ws_bytes < L.total || (reinterpret_cast<uintptr_t>(f->ws) & 255)) return GS_ERR_WORKSPACE;
  FrameTable t;
  const gs_status s = build_batch_table(f, views, nviews, cfg, t);
  if (s != GS_OK) return s;
  const cudaError_t e = launch_sequence(t, make_ptrs(L, f->ws), reinterpret_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? GS_OK : GS_ERR_CUDA;
}

gs_status gabsplat_batch_status_copy(const gs_batch_frame* f, void* dst, gs_stream stream) {
  if (!batch_sizes_ok(f) || !dst) return GS_ERR_INVALID_ARG;
  const WsLayout L = batch_layout(f);
  const WsPtrs p = make_ptrs(L, f->ws);
  // {int status, u32 epoch, u64 pairs}: the first 16 bytes of the workspace header
  return cudaMemcpyAsync(dst, p.hdr, 16, cudaMemcpyDefault, reinterpret_cast<cudaStream_t>(stream)) == cudaSuccess
             ? GS_OK
             : GS_ERR_CUDA;
}

gs_status gabsplat_batch_graph_create(const gs_batch_frame* f, const gs_config* cfg, gs_stream stream,
                                      gs_batch_graph** out) {
  if (!batch_sizes_ok(f) || !cfg || !out || !stream) return GS_ERR_INVALID_ARG;
  const WsLayout L = batch_layout(f);
  if (f->ws_bytes < L.total || (reinterpret_cast<uintptr_t>(f->ws) & 255)) return GS_ERR_WORKSPACE;
  FrameTable t;
  gs_status s = build_batch_table(f, nullptr, 0, cfg, t);   // an empty frame: every kernel returns at once
  if (s != GS_OK) return s;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const WsPtrs p = make_ptrs(L, f->ws);
  // one eager pass initialises every launcher (attributes, occupancy) outside the capture
  if (launch_sequence(t, p, st) != cudaSuccess) return GS_ERR_CUDA;
  gs_batch_graph* g = static_cast<gs_batch_graph*>(calloc(1, sizeof(gs_batch_graph)));
  if (!g) return GS_ERR_INVALID_ARG;
  cudaError_t e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    const cudaError_t le = launch_sequence(t, p, st);
    e = cudaStreamEndCapture(st, &g->graph);
    if (e == cudaSuccess && le != cudaSuccess) e = le;
  }
  size_t nn = 0;
  if (e == cudaSuccess) e = cudaGraphGetNodes(g->graph, nullptr, &nn);
  cudaGraphNode_t* nodes = nn ? static_cast<cudaGraphNode_t*>(calloc(nn, sizeof(cudaGraphNode_t))) : nullptr;
  if (e == cudaSuccess && nodes) e = cudaGraphGetNodes(g->graph, nodes, &nn);
  bool found = false;
  for (size_t i = 0; e == cudaSuccess && i < nn && !found; ++i) {
    cudaGraphNodeType ty;
    if (cudaGraphNodeGetType(nodes[i], &ty) != cudaSuccess || ty != cudaGraphNodeTypeKernel) continue;
    cudaKernelNodeParams kp;
    if (cudaGraphKernelNodeGetParams(nodes[i], &kp) != cudaSuccess) continue;
    if (kp.func == setup_kernel_fn()) {
      g->setup_node = nodes[i];
      g->setup_params = kp;
      found = true;
    }
  }
  free(nodes);
  if (e == cudaSuccess && !found) e = cudaErrorInvalidValue;
  if (e == cudaSuccess) e = cudaGraphInstantiate(&g->exec, g->graph, 0);
  if (e != cudaSuccess) {
    if (g->graph) cudaGraphDestroy(g->graph);
    free(g);
    return GS_ERR_CUDA;
  }
  g->frame = *f;
  g->cfg = *cfg;
  g->ptrs = p;
  *out = g;
  return GS_OK;
}

gs_status gabsplat_batch_graph_launch(gs_batch_graph* g, const gs_view* views, int nviews, gs_stream stream) {
  if (!g) return GS_ERR_INVALID_ARG;
  FrameTable t;
  const gs_status s = build_batch_table(&g->frame, views, nviews, &g->cfg, t);
  if (s != GS_OK) return s;
  WsPtrs p = g->ptrs;
  void* args[2] = {&t, &p};
  cudaKernelNodeParams kp = g->setup_params;
  kp.kernelParams = args;
  kp.extra = nullptr;
  cudaError_t e = cudaGraphExecKernelNodeSetParams(g->exec, g->setup_node, &kp);
  if (e == cudaSuccess) e = cudaGraphLaunch(g->exec, reinterpret_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? GS_OK : GS_ERR_CUDA;
}

void gabsplat_batch_graph_destroy(gs_batch_graph* g) {
  if (!g) return;
  if (g->exec) cudaGraphExecDestroy(g->exec);
  if (g->graph) cudaGraphDestroy(g->graph);
  free(g);
}

}  // extern "C"
