// Internal declarations shared by the rasterizer's translation units (not part of the ABI).
#pragma once

#include <utility>

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include "gabsplat.h"

namespace gs {

typedef unsigned long long u64;
typedef unsigned int u32;

constexpr int TILE = GS_TILE;
constexpr int BLOCK = 256;            // threads per CTA for every tile / chunk kernel
constexpr int CHUNK = BLOCK;          // primitives per preprocess chunk (one per thread)
constexpr int SCAN_ITEMS = 16;
constexpr int SCAN_CHUNK = BLOCK * SCAN_ITEMS;   // elements per chunk of the active-list and rank-order scans
#ifndef GS_SORT_THREADS
#define GS_SORT_THREADS 256
#endif
#ifndef GS_SORT_ITEMS
#define GS_SORT_ITEMS 16
#endif
#ifndef GS_DSORT_ITEMS
#define GS_DSORT_ITEMS 4
#endif
#ifndef GS_SORT_MIN_CTAS
#define GS_SORT_MIN_CTAS 3
#endif
constexpr int SORT_THREADS = GS_SORT_THREADS;   // >= 256: the first 256 threads own one digit each
constexpr int SORT_ITEMS = GS_SORT_ITEMS;       // keys per thread of a tile-sort partition
constexpr int DSORT_ITEMS = GS_DSORT_ITEMS;     // keys per thread of a depth-sort partition
constexpr int SORT_TILE = SORT_THREADS * (SORT_ITEMS < DSORT_ITEMS ? SORT_ITEMS : DSORT_ITEMS);   // smallest partition
constexpr int RADIX_BITS = 8;
constexpr int RADIX = 1 << RADIX_BITS;
constexpr int DPASSES = 4;     // depth-sort passes launched (depth keys have at most 32 bits)
constexpr int MAX_PASSES = 8;  // digit-pass slots: 0..3 depth sort, 4..7 tile sort
constexpr int CMASK_PLANES = 8;

// Number of floats of a projected 2D record and of a per-primitive 2D gradient row.
__host__ __device__ constexpr int round4(int x) { return (x + 3) & ~3; }
__host__ __device__ constexpr int rec_floats(int K) { return 12 + round4(3 * K); }
__host__ __device__ constexpr int g2d_floats(int K) { return round4(10 + 3 * K); }

// ------------------------------------------------------------------------------------------
// Frame description on the device: up to GS_MAX_VIEWS views, each one camera over one scene.
// A single-view frame is the special case nviews == 1.
// ------------------------------------------------------------------------------------------
struct ViewDesc {
  const float* means;
  const float* scales;
  const float* quats;
  const float* opacity;
  const void* sh;
  const void* freqs;
  const void* weights;
  float* out_rgb;
  float* out_T;
  const float* dL_drgb;
  int n, sh_degree;
  float R[9], t[3];
  float fx, fy, cx, cy, znear, zfar;
  float campos[3];
  int width, height, tiles_x, tiles_y;
  u32 prim_base;   // first record index of this view
  u32 tile_base;   // first global tile id of this view
  u64 pix_base;    // first per-pixel state index of this view
};

struct FrameTable {
  int nviews, K, storage, sh_degree;
  u32 total_prims, total_tiles;
  u64 total_pixels;
  float eps2d, alpha_max, alpha_min, T_min;
  float bg[3];
  u32 flags;                        // gs_config.flags (GS_FLAG_*)
  int tpasses;                      // tile-sort digit passes launched (fixed per workspace; host)
  int tpasses_needed;               // tile-sort passes that do work: ceil(tile bits of this frame / 8)
  int dpasses_needed;               // depth-sort passes that do work: ceil(depth_bits / 8)
  u32 depth_base;                   // float bits of the nearest depth (znear): depth keys minus this fit
  int depth_bits;                   //   in depth_bits bits
  u32 launch_prims, launch_tiles;   // host-side launch sizing (capacity of the workspace); not read on the device
  ViewDesc v[GS_MAX_VIEWS];
};

// Device-side header at the start of every workspace.
struct WsHeader {
  int status;               // gs_status of the current frame (0 = ok)
  u32 epoch;                // bumped by the setup kernel once per frame; tags look-back words
  u64 pairs;                // (tile, primitive) pairs emitted by the frame (may exceed capacity)
  u32 tile_counter_fwd;     // render_fwd tile allocator
  u32 tile_counter_bwd;     // render_bwd tile allocator
  u32 nonfinite;            // primitives culled because a projected value was not finite
  u32 sort_counter[MAX_PASSES];
  u32 timeout_site;         // which bounded wait gave up (diagnostics)
  u32 sorted_buf;           // 0: sorted pairs in keys0, 1: in keys1
  u32 n_active;             // primitives that touch at least one tile (depth ranks 0 .. n_active - 1)
  u32 fwd_exits, bwd_exits; // CTAs of the current compositing launch that have finished
  u32 masks_epoch;          // epoch of the last forward that recorded the composited-pair bits
  u32 zero_counter;         // chunks of the attribute-gradient zero-fill handed out by render_bwd
  u32 pad[10];
};

// Offsets of every region of a workspace (host-computed; all 256-byte aligned).
struct WsLayout {
  size_t header, table, records, touched, offsets, order, active, rank_of, dkeys0, dkeys1, scan_partials, rank_partials,
      keys0, keys1,
      hist, sort_status, ranges, tile_order, cmask, T_final, n_contrib, n_eval, n_reach, n_comp, grad2d, total;
  u32 n_prims, n_tiles, n_chunks, n_parts;
  u64 n_pixels, capacity;
  int K, rec_f, g2d_f;
};

// Device pointers into a workspace, passed by value to kernels.
struct WsPtrs {
  WsHeader* hdr;
  const FrameTable* tbl;
  float* records;     // [n_prims][rec_f] by depth rank (row r: primitive order[r])
  u32* touched;       // [n_prims] kept tiles per primitive
  u32* offsets;       // [n_prims] by depth rank: first pair position of the primitive of that rank
  u32* order;         // [n_prims] by depth rank: primitive index (the depth-sorted active list)
  u32* active;        // [n_prims] the active primitives in index order (emission, records and the
                      //   gradient chain run over this list: coalesced attribute access, mixed sizes)
  u32* rank_of;       // [n_prims] by primitive index: depth rank of an active primitive
  u64* dkeys0;        // [n_prims] depth-sort keys (depth bits - depth_base) << 32 | primitive; dkeys1 also
  u64* dkeys1;        //   holds each active primitive's key at its primitive index before the scan
  u64* scan_partials;   // [n_chunks] per-chunk sums of the active-list scan
  u64* rank_partials;   // [n_chunks] per-chunk sums of the rank-order scan
  u64* keys0;         // [capacity] pairs tile << 32 | depth rank (emission order, then sort ping-pong)
  u64* keys1;
  u32* hist;          // [MAX_PASSES][RADIX]
  u64* sort_status;   // [n_parts][RADIX]
  uint2* ranges;      // [n_tiles]
  u32* tile_order;    // [n_tiles] tiles by descending pair count (the compositing kernels' schedule)
  u32* cmask;         // [CMASK_PLANES][cmask_plane] per compositing warp slot: bit (pos & 31) of word
                      // (pos >> 5) + tile set if a pixel of that warp composited the pair at sorted position pos
  float* T_final;     // [n_pixels]
  u32* n_contrib;     // [n_pixels]
  u32* n_eval;        // [n_pixels] pairs the forward pass evaluated per pixel
  u32* n_reach;       // [n_pixels] of those, pairs that passed the footprint test (o G >= alpha_min)
  u32* n_comp;        // [n_pixels] pairs composited
  float* grad2d;      // [n_prims][g2d_f] by depth rank
  u64 capacity;
  u32 n_chunks, n_parts;
  u32 cmask_plane;     // words per plane: capacity / 32 + tiles + 2 (each tile owns whole words)
};

WsLayout make_layout(u32 n_prims, int K, u32 n_tiles, u64 n_pixels, u64 capacity);
int tile_passes(u32 ntiles);
int tile_bits(u32 ntiles);
void set_depth_window(FrameTable& t, float znear_min, float zfar_max);

WsPtrs make_ptrs(const WsLayout& L, void* ws);

// ------------------------------------------------------------------------------------------
// Decoupled look-back words: [63:62] flag, [61:40] tag, [39:0] value.
// ------------------------------------------------------------------------------------------
constexpr u64 LB_FLAG_AGG = 1ull;
constexpr u64 LB_FLAG_PREFIX = 2ull;
__device__ __forceinline__ u64 lb_pack(u64 flag, u32 tag, u64 value) {
  return (flag << 62) | ((u64)(tag & 0x3FFFFFu) << 40) | (value & 0xFFFFFFFFFFull);
}
__device__ __forceinline__ u32 lb_flag(u64 w) { return (u32)(w >> 62); }
__device__ __forceinline__ u32 lb_tag(u64 w) { return (u32)(w >> 40) & 0x3FFFFFu; }
__device__ __forceinline__ u64 lb_value(u64 w) { return w & 0xFFFFFFFFFFull; }

__device__ __forceinline__ u64 ld_relaxed(const u64* p) {
  u64 v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_relaxed(u64* p, u64 v) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ u64 global_timer_ns() {
  u64 t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}

// Every spin-wait gives up after this long (or this many polls) and sets GS_ERR_TIMEOUT.
constexpr u64 SPIN_LIMIT_NS = 1000000000ull;   // 1 s
constexpr u32 SPIN_LIMIT_POLLS = 1u << 24;

__device__ __forceinline__ void set_status(WsHeader* hdr, int s);

#ifndef GS_LB_WINDOW
#define GS_LB_WINDOW 4
#endif
constexpr int LB_WINDOW = GS_LB_WINDOW;   // look-back words read per step

// Decoupled look-back walk of partition `part` (one thread): adds the published values of
// partitions part - 1, part - 2, ... (word of partition j at status[j * stride]) back to the nearest
// inclusive prefix and returns that exclusive prefix.  LB_WINDOW predecessors are read per step as
// independent loads (one memory latency); consumption stops at the first word not yet published
// for this tag, which is polled again.  Partition 0 always publishes a prefix.  Bounded: after the
// spin limit it sets GS_ERR_TIMEOUT (site `site`) and returns what it has.
__device__ __forceinline__ u64 lookback_walk(const u64* status, u64 stride, u32 part, u32 tag, WsHeader* hdr,
                                             u32 site) {
  const u32 tag22 = tag & 0x3FFFFFu;
  u64 excl = 0;
  u32 pi = part;   // partitions pi - 1, pi - 2, ... are still to be added
  u32 polls = 0;
  const u64 t0 = global_timer_ns();
  for (;;) {
    u64 w[LB_WINDOW];
#pragma unroll
    for (int j = 0; j < LB_WINDOW; ++j) w[j] = (u32)j < pi ? ld_relaxed(status + (u64)(pi - 1 - j) * stride) : 0ull;
    u32 used = 0;
#pragma unroll
    for (int j = 0; j < LB_WINDOW; ++j) {
      if (used != (u32)j || (u32)j >= pi) break;   // an earlier word stopped the walk
      if (lb_flag(w[j]) == 0 || lb_tag(w[j]) != tag22) break;
      excl += lb_value(w[j]);
      if (lb_flag(w[j]) == LB_FLAG_PREFIX) return excl;
      ++used;
    }
    pi -= used;
    if (used == 0) {
      if (++polls > SPIN_LIMIT_POLLS || ((polls & 1023u) == 0 && global_timer_ns() - t0 > SPIN_LIMIT_NS)) {
        hdr->timeout_site = site;
        set_status(hdr, GS_ERR_TIMEOUT);
        return excl;
      }
      __nanosleep(20);
    }
  }
}

__device__ __forceinline__ void set_status(WsHeader* hdr, int s) { atomicCAS(&hdr->status, 0, s); }
__device__ __forceinline__ int read_status(const WsHeader* hdr) {
  return *((volatile const int*)&hdr->status);
}

// Which view does a global primitive / tile index belong to (nviews <= 16, linear scan).
__device__ __forceinline__ int view_of_prim(const FrameTable* t, u32 gi) {
  int v = 0;
  const int nv = t->nviews;
  while (v + 1 < nv && gi >= t->v[v + 1].prim_base) ++v;
  return v;
}
__device__ __forceinline__ int view_of_tile(const FrameTable* t, u32 tile) {
  int v = 0;
  const int nv = t->nviews;
  while (v + 1 < nv && tile >= t->v[v + 1].tile_base) ++v;
  return v;
}

template <int STORAGE>
__device__ __forceinline__ float load_attr(const void* p, size_t i) {
  if (STORAGE == GS_BF16) return __bfloat162float(reinterpret_cast<const __nv_bfloat16*>(p)[i]);
  return __ldg(reinterpret_cast<const float*>(p) + i);
}

// Row `row` of N values ([rows][N] in the storage type) as float32, with the widest loads that the
// row length and the address allow.
template <int STORAGE, int N>
__device__ __forceinline__ void load_row(const void* p, size_t row, float* out) {
  if (N == 0) return;
  if (STORAGE == GS_BF16) {
    const __nv_bfloat16* src = reinterpret_cast<const __nv_bfloat16*>(p) + row * N;
    if (N % 2 == 0 && (reinterpret_cast<uintptr_t>(src) & 3) == 0) {
#pragma unroll
      for (int i = 0; i < N / 2; ++i) {
        const float2 f = __bfloat1622float2(reinterpret_cast<const __nv_bfloat162*>(src)[i]);
        out[2 * i] = f.x;
        out[2 * i + 1] = f.y;
      }
    } else {
#pragma unroll
      for (int i = 0; i < N; ++i) out[i] = __bfloat162float(src[i]);
    }
  } else {
    const float* src = reinterpret_cast<const float*>(p) + row * N;
    if (N % 4 == 0 && (reinterpret_cast<uintptr_t>(src) & 15) == 0) {
#pragma unroll
      for (int i = 0; i < N / 4; ++i) {
        const float4 t = __ldg(reinterpret_cast<const float4*>(src) + i);
        out[4 * i] = t.x; out[4 * i + 1] = t.y; out[4 * i + 2] = t.z; out[4 * i + 3] = t.w;
      }
    } else if (N % 2 == 0 && (reinterpret_cast<uintptr_t>(src) & 7) == 0) {
#pragma unroll
      for (int i = 0; i < N / 2; ++i) {
        const float2 t = __ldg(reinterpret_cast<const float2*>(src) + i);
        out[2 * i] = t.x; out[2 * i + 1] = t.y;
      }
    } else {
#pragma unroll
      for (int i = 0; i < N; ++i) out[i] = __ldg(src + i);
    }
  }
}

// N float32 values to row `row` of p ([rows][N]), with the widest stores the row and address allow.
template <int N>
__device__ __forceinline__ void store_row(float* p, size_t row, const float* v) {
  if (N == 0) return;
  float* dst = p + row * N;
  if (N % 4 == 0 && (reinterpret_cast<uintptr_t>(dst) & 15) == 0) {
#pragma unroll
    for (int i = 0; i < N / 4; ++i)
      reinterpret_cast<float4*>(dst)[i] = make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
  } else if (N % 2 == 0 && (reinterpret_cast<uintptr_t>(dst) & 7) == 0) {
#pragma unroll
    for (int i = 0; i < N / 2; ++i) reinterpret_cast<float2*>(dst)[i] = make_float2(v[2 * i], v[2 * i + 1]);
  } else {
#pragma unroll
    for (int i = 0; i < N; ++i) dst[i] = v[i];
  }
}

// The 3 nsh SH coefficients of primitive k ([k][nsh][3] in the storage type) as float32.  A full
// degree-3 row (192 B in float32, 96 B in BF16) is read with 16-byte loads, all issued before use.
template <int STORAGE>
__device__ __forceinline__ void load_sh_row(const void* sh, size_t k, int nsh, float* c) {
  const size_t base = k * (size_t)nsh * 3;
  if (nsh == 16 && (reinterpret_cast<uintptr_t>(sh) & 15) == 0) {
    if (STORAGE == GS_BF16) {
      const uint4* src = reinterpret_cast<const uint4*>(reinterpret_cast<const __nv_bfloat16*>(sh) + base);
      uint4 t[6];
#pragma unroll
      for (int i = 0; i < 6; ++i) t[i] = __ldg(src + i);
#pragma unroll
      for (int i = 0; i < 6; ++i) {
        const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&t[i]);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const float2 f = __bfloat1622float2(h[j]);
          c[8 * i + 2 * j] = f.x;
          c[8 * i + 2 * j + 1] = f.y;
        }
      }
    } else {
      const float4* src = reinterpret_cast<const float4*>(reinterpret_cast<const float*>(sh) + base);
      float4 t[12];
#pragma unroll
      for (int i = 0; i < 12; ++i) t[i] = __ldg(src + i);
#pragma unroll
      for (int i = 0; i < 12; ++i) {
        c[4 * i] = t[i].x; c[4 * i + 1] = t[i].y; c[4 * i + 2] = t[i].z; c[4 * i + 3] = t[i].w;
      }
    }
    return;
  }
#pragma unroll
  for (int i = 0; i < 48; ++i)
    if (i < 3 * nsh) c[i] = load_attr<STORAGE>(sh, base + i);
}

// ------------------------------------------------------------------------------------------
// Programmatic dependent launch.  The kernels of the path are launched with programmatic stream
// serialization, so a kernel's CTAs may be scheduled while the kernel before it in the stream is
// still draining.  Each kernel begins with pdl_begin(): griddepcontrol.wait blocks until the
// predecessor grid has completed and its memory operations are visible (a no-op when the kernel
// was launched without the attribute), and launch_dependents then lets the successor be
// scheduled.  Kernels therefore still run one after another in stream order; what overlaps is the
// successor's launch and scheduling with the predecessor's tail.  GS_PDL=0 launches plainly.
// ------------------------------------------------------------------------------------------
#ifndef GS_PDL
#define GS_PDL 1
#endif
// Launch groups that use it (bits): 0 setup, binning and the active-list scan; 1 depth-sort passes;
// 2 rank-order scan; 3 emission and records; 4 tile sort, ranges and schedule; 5 compositing
// kernels; 6 losses; 7 attribute-gradient chain; 8 density control.  Measured at 1.5M primitives,
// 1600x1064: every group but the rank-order scan 1.970 ms per training step, no group 1.982, all
// groups 1.992 (the rank-order scan's two launches cost 22 us under it), so that group is left out.
#ifndef GS_PDL_MASK
#define GS_PDL_MASK 0x1FB
#endif
enum PdlGroup { PDL_BIN = 0, PDL_DSORT, PDL_RANK, PDL_EMIT, PDL_TSORT, PDL_RENDER, PDL_LOSS, PDL_PBWD, PDL_DENSIFY };
__device__ __forceinline__ void pdl_begin() {
#if GS_PDL == 2
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  asm volatile("griddepcontrol.wait;" ::: "memory");
#else
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
#endif
}

template <int GROUP, typename... Params, typename... Args>
static inline cudaError_t launch_pdl(void (*kernel)(Params...), dim3 grid, dim3 block, size_t smem,
                                     cudaStream_t stream, Args&&... args) {
  constexpr bool on = GS_PDL && ((GS_PDL_MASK >> GROUP) & 1);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = on ? 1 : 0;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

// ------------------------------------------------------------------------------------------
// Launch helpers (defined in the kernel translation units).
// ------------------------------------------------------------------------------------------
struct Launch {
  int sm_count;
  cudaStream_t stream;
};
int device_sm_count();

cudaError_t launch_setup(const FrameTable& tbl, const WsPtrs& p, const Launch& L);
cudaError_t launch_preprocess(const FrameTable& tbl, const WsPtrs& p, const Launch& L);
cudaError_t launch_depth_sort(const FrameTable& tbl, const WsPtrs& p, const Launch& L);
cudaError_t launch_bin_sort(const FrameTable& tbl, const WsPtrs& p, const Launch& L);
// masks: record the composited-pair bits the backward pass reads (off for forward-only rendering)
// stats: also write the per-pixel work counters n_eval, n_reach, n_comp (only with masks)
cudaError_t launch_render_fwd(const FrameTable& tbl, const WsPtrs& p, float* out_rgb, float* out_T, const Launch& L,
                              bool masks, bool stats = false);
cudaError_t launch_render_freq_map(const FrameTable& tbl, const WsPtrs& p, float* out_map, const Launch& L);
// Zero-fill of the attribute gradients carried out by the compositing backward: that kernel is
// bound by instruction issue and the fill by HBM writes, so the fill runs in its shadow.  The
// arrays are cut into chunks of ZERO_CHUNK floats; a CTA takes `quota` chunks after each tile and
// the rest once the tile queue is empty.
#ifndef GS_ZERO_SPREAD_PCT
#define GS_ZERO_SPREAD_PCT 50   // the fill is handed out by the time this share of the tiles is taken
#endif
constexpr int ZERO_ARRAYS = 8;
constexpr u32 ZERO_CHUNK = 4096;
struct ZeroJob {
  float* a[ZERO_ARRAYS];
  u64 n[ZERO_ARRAYS];          // floats of each array (0 for a NULL pointer)
  u32 base[ZERO_ARRAYS + 1];   // first chunk of each array; base[ZERO_ARRAYS] = total chunks
  u32 quota;                   // chunks per tile; 0: no fill
};
// The zero-fill of every array of g (n primitives, K Gabor components, nsh SH coefficients per
// channel), spread so that it is handed out by the time GS_ZERO_SPREAD_PCT % of the ntiles tiles
// are taken.
ZeroJob make_zero_job(const gs_prim_grads& g, int n, int K, int nsh, u32 ntiles);

// z: NULL, or a zero-fill for the kernel to carry out.
cudaError_t launch_render_bwd(const FrameTable& tbl, const WsPtrs& p, const float* dL_drgb, const ZeroJob* z,
                              const Launch& L);
// prezeroed: the gradients of primitives that reach no tile are already zero (a ZeroJob of the
// same arrays ran in this frame's render_bwd), so only the active primitives' rows are written.
cudaError_t launch_preprocess_bwd(const FrameTable& tbl, const WsPtrs& p, const gs_prim_grads& g, bool prezeroed,
                                  const Launch& L);
cudaError_t launch_loss(const float* img, const float* tgt, long long count, int kind, double* loss_out, float* dL,
                        double* partials, int nblocks, cudaStream_t s);
size_t l1_dssim_partials(int C, int H, int W);
cudaError_t launch_densify_accumulate(const u32* touched, int n, const float* grad, float* acc, float* den,
                                      int sm_count, cudaStream_t s);
cudaError_t launch_l1_dssim(const float* img, const float* tgt, int C, int H, int W, float lambda, double* loss_out,
                            float* dL, double* partials, cudaStream_t s);

}  // namespace gs
