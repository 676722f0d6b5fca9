// Per-tile compositing of the 2D Gabor primitives (Sec. 3.3.2 Eq. 9, Sec. 3.3.3 Eq. 10) and its
// reverse-order adjoint.  Both kernels run independent warps: a warp pulls one 8x8 footprint of a
// 16x16 tile at a time from an atomic counter (tiles with the longest pair lists first) and stages
// pair records into its own shared-memory rows.  The forward walks the tile's depth-sorted pairs
// front to back until its pixels saturate; the backward walks, back to front, only the pairs the
// forward recorded as composited in that footprint.  Envelope, bank and alpha are evaluated with
// explicit rounding intrinsics in both, so the backward reproduces the forward's decisions exactly.
#include <type_traits>

#include "common.cuh"

namespace gs {

// Unroll factors of the pair loops: consecutive pairs' independent arithmetic (phases, cosines,
// exponentials) can then overlap the previous pair's blend.  Measured at 1.5M primitives,
// 1600x1064: forward 4 at 8 CTAs per SM 0.459 ms (1: 0.493 at 9 CTAs, 8: 0.468, 32: 0.989, the
// instruction cache overflowing); backward 2 at 6 CTAs per SM 0.732 ms (1: 0.742 at 7 CTAs; 2 at 7
// CTAs: 0.748; 4: 0.796).
#ifndef GS_FWD_UNROLL
#define GS_FWD_UNROLL 4
#endif
constexpr int FWD_UNROLL = GS_FWD_UNROLL;
// Unroll factor of the backward's pair loop.
#ifndef GS_BWD_UNROLL
#define GS_BWD_UNROLL 2
#endif
constexpr int BWD_UNROLL = GS_BWD_UNROLL;

constexpr float LOG2E = 1.4426950408889634f;
constexpr float TWO_PI = 6.283185307179586f;
constexpr float INV_TWO_PI = 0.15915494309189535f;

// Shared-memory record (floats), staged by a warp for its footprint: {mu_x, mu_y, A', B'},
// {C', thr, o, 1 - sum w}, {r, g, b, fast}, {2 pi f2D_0x, 2 pi f2D_0y, ...}, {w_0 ...};
// A' = -a/2 log2 e, B' = -b log2 e, C' = -c/2 log2 e so that G = 2^(A' dx^2 + B' dx dy + C' dy^2);
// thr = log2(alpha_min / o): o G < alpha_min <=> power < thr, and since the filter bank is <= 1
// (weights >= 0) such pairs have alpha < alpha_min: skipped early.  fast = 1 when every
// |f2D_i . (x - mu)| over the pixel centres x of the footprint is within FAST_PHASE_CYCLES, so the
// phase needs no range reduction; the forward and the backward stage the same footprints, so both
// evaluate the bank the same way.
template <int K>
struct SRec {
  static constexpr int F = rec_floats(K);
  static constexpr int F4 = F / 4;
};
// Largest |phase| (cycles) taken by cos / sin without range reduction: the hardware approximation's
// error grows with the argument (measured on the B300: about 4e-7 within half a cycle, 1.3e-6
// within two cycles).
constexpr float FAST_PHASE_CYCLES = 2.0f;

// Stages one global record for a footprint whose pixel centres span [lo.x, hi.x] x [lo.y, hi.y]:
// the f2D values are scaled by 2 pi, and the footprint's fast flag replaces slot 11.
template <int K>
__device__ __forceinline__ void stage_record(const float* __restrict__ rec, float4* dst, float alpha_min, float2 lo,
                                             float2 hi) {
  const float4* src = reinterpret_cast<const float4*>(rec);
  const float4 h0 = __ldg(src), h1 = __ldg(src + 1), h2 = __ldg(src + 2);
  const float o = h1.y;
  dst[0] = make_float4(h0.x, h0.y, -0.5f * LOG2E * h0.z, -LOG2E * h0.w);
  dst[1] = make_float4(-0.5f * LOG2E * h1.x, o > 0.f ? log2f(alpha_min / o) : 3.0e38f, o, h1.z);
  const float ax = fmaxf(fabsf(lo.x - h0.x), fabsf(hi.x - h0.x)), ay = fmaxf(fabsf(lo.y - h0.y), fabsf(hi.y - h0.y));
  float bound = 0.f;   // the largest |f2D_i . (x - mu)| over the footprint, in cycles
#pragma unroll
  for (int i = 0; i < SRec<K>::F4 - 3; ++i) {
    float4 t = __ldg(src + 3 + i);
    // floats 0 .. 2K - 1 after the colour are f2D (scaled); the weights follow (for odd K in the
    // same float4 as the last component)
    if (4 * i + 1 < 2 * K) bound = fmaxf(bound, fabsf(t.x) * ax + fabsf(t.y) * ay);
    if (4 * i + 3 < 2 * K) bound = fmaxf(bound, fabsf(t.z) * ax + fabsf(t.w) * ay);
    if (4 * i + 0 < 2 * K) t.x = __fmul_rn(TWO_PI, t.x);
    if (4 * i + 1 < 2 * K) t.y = __fmul_rn(TWO_PI, t.y);
    if (4 * i + 2 < 2 * K) t.z = __fmul_rn(TWO_PI, t.z);
    if (4 * i + 3 < 2 * K) t.w = __fmul_rn(TWO_PI, t.w);
    dst[3 + i] = t;
  }
  dst[2] = make_float4(h2.x, h2.y, h2.z, bound <= FAST_PHASE_CYCLES ? 1.f : 0.f);
}

// Frequency features of one record: sum_i w_i |f2D_i|, sum_i w_i |f2D_i,x|, sum_i w_i |f2D_i,y|.
template <int K>
__device__ __forceinline__ float4 frequency_features(const float* __restrict__ rec) {
  float m = 0.f, mx = 0.f, my = 0.f;
#pragma unroll
  for (int i = 0; i < K; ++i) {
    const float fx = __ldg(rec + 12 + 2 * i), fy = __ldg(rec + 13 + 2 * i), w = __ldg(rec + 12 + 2 * K + i);
    m = fmaf(w, sqrtf(fx * fx + fy * fy), m);
    mx = fmaf(w, fabsf(fx), mx);
    my = fmaf(w, fabsf(fy), my);
  }
  return make_float4(m, mx, my, 0.f);
}

__device__ __forceinline__ float rcp_approx(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// Two pixels' values in one register pair.  The packed FP32 instructions of sm_100 and later
// (__ffma2_rn, __fmul2_rn, __fadd2_rn) work on both halves with one issue and round each half
// exactly as the scalar instruction does, so packed and scalar evaluation give the same bits.
__device__ __forceinline__ float2 f2(float v) { return make_float2(v, v); }

// Exponent (log2 domain) of the 2D Gaussian at offset (dx, dy).
__device__ __forceinline__ float gauss_power(const float4& h0, const float4& h1, float dx, float dy) {
  return __fmaf_rn(dx, __fmaf_rn(h0.z, dx, __fmul_rn(h0.w, dy)), __fmul_rn(__fmul_rn(h1.x, dy), dy));
}

// Envelope exponents of a thread's PPT pixels (rows y .. y + PPT - 1 of one column, offsets dx and
// dy[q] from the mean).  Two rows are evaluated directly, both in one packed instruction stream;
// more rows follow row q by the recurrence pw(dy + 1) = pw(dy) + B' dx + C' (2 dy + 1).  The
// forward and the backward both use it, so they take the same decisions.
template <int PPT>
__device__ __forceinline__ void pixel_powers(const float4& h0, const float4& h1, float dx, float dy0, float* dy,
                                             float* pw) {
  dy[0] = dy0;
  if constexpr (PPT == 2) {
    dy[1] = __fadd_rn(dy0, 1.f);
    const float2 d = make_float2(dy[0], dy[1]);
    const float2 e = __ffma2_rn(f2(dx), __ffma2_rn(f2(h0.z), f2(dx), __fmul2_rn(f2(h0.w), d)),
                                __fmul2_rn(__fmul2_rn(f2(h1.x), d), d));   // gauss_power of each row
    pw[0] = e.x;
    pw[1] = e.y;
    return;
  }
  pw[0] = gauss_power(h0, h1, dx, dy0);
  const float bdx = __fmul_rn(h0.w, dx);
#pragma unroll
  for (int q = 1; q < PPT; ++q) {
    dy[q] = __fadd_rn(dy[q - 1], 1.f);
    pw[q] = __fadd_rn(pw[q - 1], __fmaf_rn(h1.x, __fmaf_rn(2.f, dy[q - 1], 1.f), bdx));
  }
}

// Phase 2 pi f2D . d (radians) of a thread's first pixel from the staged (2 pi f2D_x, 2 pi f2D_y).
// With more than two rows per thread each further row adds 2 pi f2D_y; two rows are evaluated
// directly (row_phases2).
__device__ __forceinline__ float raw_phase(float Fx, float Fy, float dx, float dy) {
  return __fmaf_rn(Fx, dx, __fmul_rn(Fy, dy));
}

// Phases of both rows of a thread's column, each as raw_phase gives it for its own offset.
__device__ __forceinline__ float2 row_phases2(float Fx, float Fy, float dx, const float* dy) {
  return __ffma2_rn(f2(Fx), f2(dx), __fmul2_rn(f2(Fy), make_float2(dy[0], dy[1])));
}

// FAST: the phase as it is; otherwise reduced to [-pi, pi] through cycles,
// cos(2 pi t) = cos(2 pi (t - rint(t))).
template <bool FAST>
__device__ __forceinline__ float reduced_angle(float th) {
  if (FAST) return th;
  const float t = __fmul_rn(th, INV_TWO_PI);
  return __fmul_rn(TWO_PI, __fsub_rn(t, rintf(t)));
}

// reduced_angle on both halves: t - rint(t) = t + rint(-t) is exact, so this equals the scalar form.
template <bool FAST>
__device__ __forceinline__ float2 reduced_angle2(float2 th) {
  if (FAST) return th;
  const float2 t = __fmul2_rn(th, f2(INV_TWO_PI));
  return __fmul2_rn(f2(TWO_PI), __fadd2_rn(t, make_float2(rintf(-t.x), rintf(-t.y))));
}

// Filter bank (1 - sum w) + sum w_i cos(2 pi f2D_i . d)  (Sec. 3.3.2, Eq. 9) from the phases.
template <int K, bool FAST>
__device__ __forceinline__ float filter_bank(const float* th, const float* w, float w0) {
  float bank = w0;
#pragma unroll
  for (int i = 0; i < K; ++i) bank = __fmaf_rn(w[i], __cosf(reduced_angle<FAST>(th[i])), bank);
  return bank;
}

// Pixels per thread of the compositing kernels: a thread owns PPT vertically adjacent pixels of
// its tile column, so each shared-memory record load and (backward) each warp reduction of the
// per-pair gradients serves PPT pixels.  CTAs have 256 / PPT threads.
#ifndef GS_PPT_FWD
#define GS_PPT_FWD 2
#endif
#ifndef GS_PPT_BWD
#define GS_PPT_BWD 2
#endif
static_assert(GS_PPT_FWD == GS_PPT_BWD, "the backward reads the forward's per-warp composited-pair bits: same warp footprints");

// Warp footprint inside the 16x16 tile: 1 = 8 pixels wide and 4 PPT rows high (two warp columns),
// 0 = the full tile width and 2 PPT rows high.  A compact footprint means fewer warps overlap a
// small splat, so fewer warps run the per-pair gradient block and its reduction (8x8 at PPT = 2:
// 5% less time in the backward than 16x4 at 1.5M primitives, 1600x1064).
#ifndef GS_WARP_SQUARE
#define GS_WARP_SQUARE 1
#endif

// Resident CTAs per SM the compositing kernels are compiled for (0: the compiler's choice).  With
// the pair loops unrolled (above), the backward's warp walk with the two-pixel packed adjoint runs
// at 6 CTAs of 128 threads per SM (80 registers, a 4-byte spill) and the forward at 8 (64
// registers, no spill).  Without the unroll the backward measured 0.750 ms at 7 CTAs (72
// registers), 0.760 at 6 and 0.767 at 5; the forward 0.503 at 9 (56 registers) and 0.507 at the
// compiler's own 48 registers.  The packed adjoint holds both pixels' cosines and sines, so above
// K = 4 it runs at GS_BWD_MIN_CTAS_HIGHK (K = 8: 96 registers, a 16-byte spill at 5 CTAs per SM;
// render_bwd 1.280 ms at 3M primitives, 1920x1080, against 1.338 at 4 CTAs and 1.487 for the
// per-pixel adjoint, which K above GS_BWD_PACKED_MAX_K and PPT other than 2 use, at 4 CTAs).
#ifndef GS_FWD_MIN_CTAS
#define GS_FWD_MIN_CTAS 8
#endif
#ifndef GS_BWD_MIN_CTAS
#define GS_BWD_MIN_CTAS 6
#endif
#ifndef GS_BWD_MIN_CTAS_HIGHK
#define GS_BWD_MIN_CTAS_HIGHK 5   // the packed adjoint above K = 4
#endif
#ifndef GS_BWD_UNROLL_HIGHK
#define GS_BWD_UNROLL_HIGHK 2
#endif
#ifndef GS_BWD_PACKED_MAX_K
#define GS_BWD_PACKED_MAX_K 8
#endif
#if GS_FWD_MIN_CTAS
#define GS_FWD_BOUNDS __launch_bounds__(BLOCK / PPT, GS_FWD_MIN_CTAS)
#else
#define GS_FWD_BOUNDS __launch_bounds__(BLOCK / PPT)
#endif
#if GS_BWD_MIN_CTAS
#define GS_BWD_BOUNDS \
  __launch_bounds__(BLOCK / PPT, K <= 4 ? GS_BWD_MIN_CTAS : K <= GS_BWD_PACKED_MAX_K ? GS_BWD_MIN_CTAS_HIGHK : 4)
#else
#define GS_BWD_BOUNDS __launch_bounds__(BLOCK / PPT)
#endif

// Called by thread 0 of every CTA after it has left its tile loop: the last CTA of the launch
// resets the tile allocator (and counter2, the backward's zero-fill chunk counter, if given), so
// each compositing launch of a frame starts from tile 0.
__device__ __forceinline__ void release_tile_counter(u32* counter, u32* exits, u32* counter2 = nullptr) {
  __threadfence();
  if (atomicAdd(exits, 1u) == gridDim.x - 1) {
    *counter = 0;
    if (counter2) *counter2 = 0;
    *exits = 0;
  }
}

// First pixel (x, y) of thread tid in tile (tx, ty); the thread owns rows y .. y + PPT - 1.
template <int PPT>
__device__ __forceinline__ int2 thread_pixel(int tx, int ty, int tid) {
#if GS_WARP_SQUARE
  const int w = tid >> 5, lane = tid & 31;
  return make_int2(tx * TILE + (w & 1) * 8 + (lane & 7), ty * TILE + (w >> 1) * (4 * PPT) + (lane >> 3) * PPT);
#else
  return make_int2(tx * TILE + (tid & (TILE - 1)), ty * TILE + (tid >> 4) * PPT);
#endif
}

// Pixel-centre bounds (lo and hi corners) of the warp footprint holding lane `lane`, whose first
// pixel centre is (fpx, fpy0) (thread_pixel's layout).
template <int PPT>
__device__ __forceinline__ void footprint_bounds(float fpx, float fpy0, int lane, float2& lo, float2& hi) {
#if GS_WARP_SQUARE
  constexpr int FW = 8, FH = 4 * PPT;
  lo = make_float2(fpx - (float)(lane & 7), fpy0 - (float)((lane >> 3) * PPT));
#else
  constexpr int FW = TILE, FH = 2 * PPT;
  lo = make_float2(fpx - (float)(lane & 15), fpy0 - (float)((lane >> 4) * PPT));
#endif
  hi = make_float2(lo.x + (float)(FW - 1), lo.y + (float)(FH - 1));
}

// The forward with independent warps.  A task is one warp footprint (8x8 pixels at PPT = 2) of one
// tile, tiles in the order of tile_order (longest pair lists first).  A warp stages the tile's
// pairs into its own shared-memory rows one 32-position word of the sorted list at a time (the
// unit of the composited-pair bits), composites them, and stops once every pixel of its footprint
// is saturated; no CTA barrier sits on the walk, so a warp that is done moves on to its next task
// instead of waiting for the others of its CTA.
// FMAP: composite the frequency features of each primitive (sum_i w_i |f2D_i|, sum_i w_i |f2D_i,x|,
// sum_i w_i |f2D_i,y|, cycles per pixel) in place of its colour, with no background.
// MASKS: record per warp which pairs its pixels composited (for the backward pass); forward-only
// uses (serving, frequency maps) skip it and keep the per-thread early exit.
// STATS: also write the per-pixel work counters (pairs evaluated, reached and composited), which
// only the work accounting and the tests read.
template <int K, int PPT, bool FMAP, bool MASKS, bool STATS>
__global__ void GS_FWD_BOUNDS k_render_fwd_w(WsPtrs p, float* out_rgb, float* out_T) {
  pdl_begin();
  constexpr int NW = BLOCK / PPT / 32;   // warps per CTA, and warp footprints per tile
  constexpr int F4 = SRec<K>::F4;
  extern __shared__ __align__(16) float4 smem4[];
  const int lane = threadIdx.x & 31;
  float4* s_rec = smem4 + (threadIdx.x >> 5) * 32 * F4;   // [32][F4] this warp's staged records
  WsHeader* hdr = p.hdr;
  if (read_status(hdr) != 0) return;
  if (MASKS && blockIdx.x == 0 && threadIdx.x == 0) hdr->masks_epoch = hdr->epoch;   // bits of this frame
  const FrameTable* tbl = p.tbl;
  // sorted pairs tile << 32 | depth rank; the rank is the record (and grad2d) row
  const u64* __restrict__ pairs = (tbl->tpasses_needed & 1) ? p.keys1 : p.keys0;
  const u32 ntiles = tbl->total_tiles;
  const float amax = tbl->alpha_max, amin = tbl->alpha_min, Tmin = tbl->T_min;
  for (;;) {
    u32 slot = 0;
    if (lane == 0) slot = atomicAdd(&hdr->tile_counter_fwd, 1u);
    slot = __shfl_sync(0xffffffffu, slot, 0);
    if (slot >= ntiles * (u32)NW) break;   // warp-uniform
    const u32 tile = p.tile_order[slot / NW];
    const int quad = (int)(slot % NW);
    const int v = view_of_tile(tbl, tile);
    const ViewDesc& V = tbl->v[v];
    const u32 local = tile - V.tile_base;
    const int tx = (int)(local % (u32)V.tiles_x), ty = (int)(local / (u32)V.tiles_x);
    const int2 pxy = thread_pixel<PPT>(tx, ty, quad * 32 + lane);
    const int px = pxy.x, py0 = pxy.y;
    const uint2 rg = p.ranges[tile];
    const float fpx = (float)px + 0.5f, fpy0 = (float)py0 + 0.5f;
    float T[PPT], C0[PPT], C1[PPT], C2[PPT];
    u32 last[PPT], evaluated[PPT], reached[PPT], composited[PPT];
    bool done[PPT];
    bool tdone = true;
#pragma unroll
    for (int q = 0; q < PPT; ++q) {
      T[q] = 1.f; C0[q] = C1[q] = C2[q] = 0.f;
      last[q] = 0; evaluated[q] = rg.y - rg.x; reached[q] = 0; composited[q] = 0;
      done[q] = !(px < V.width && py0 + q < V.height);
      tdone = tdone && done[q];
    }
    // composited-pair bits of this footprint, one word per 32 sorted positions (each tile owns
    // whole words), for the backward pass to skip the pairs no pixel of the warp composited
    u32* cplane = p.cmask + (size_t)quad * p.cmask_plane;
    for (u32 start = rg.x; start < rg.y && !__all_sync(0xffffffffu, tdone);) {
      const u32 end = min(rg.y, (start | 31u) + 1u);   // the rest of start's word
      const int cnt = (int)(end - start);
      if (lane < cnt) {
        const float* rec = p.records + (size_t)(u32)pairs[start + (u32)lane] * rec_floats(K);
        float2 flo, fhi;
        footprint_bounds<PPT>(fpx, fpy0, lane, flo, fhi);
        stage_record<K>(rec, s_rec + lane * F4, amin, flo, fhi);
        if (FMAP) {   // the frequency features take the colour's place; the fast flag stays
          float4 ff = frequency_features<K>(rec);
          ff.w = s_rec[lane * F4 + 2].w;
          s_rec[lane * F4 + 2] = ff;
        }
      }
      __syncwarp();
      u32 lbits = 0;
#pragma unroll FWD_UNROLL
      for (int j = 0; j < cnt; ++j) {
        if (!MASKS && tdone) break;   // with the bits every lane walks the word to its end
        const float4* r = s_rec + j * F4;
        const float4 h0 = r[0], h1 = r[1];
        const bool fast = reinterpret_cast<const float*>(r)[11] != 0.f;   // the same for every lane
        const float dx = __fsub_rn(fpx, h0.x);
        float dyq[PPT], pwq[PPT];
        pixel_powers<PPT>(h0, h1, dx, __fsub_rn(fpy0, h0.y), dyq, pwq);
        bool reach[PPT], any = false;
#pragma unroll
        for (int q = 0; q < PPT; ++q) {
          reach[q] = !done[q] && pwq[q] >= h1.y;
          any = any || reach[q];
        }
        bool comp = false;
        // the per-pixel work, instantiated for records with and without phase reduction
        auto pixels = [&](auto fast_tag) {
          const float* fr = reinterpret_cast<const float*>(r + 3);
          if constexpr (PPT == 2) {
            // both pixels at once in packed FP32 (bit-identical to the per-pixel form below); the
            // envelope, bank and alpha of a pixel that is not reached are computed and discarded
            float2 thp[K > 0 ? K : 1];
#pragma unroll
            for (int i = 0; i < K; ++i) thp[i] = row_phases2(fr[2 * i], fr[2 * i + 1], dx, dyq);
            const float2 G = make_float2(ex2_approx(pwq[0]), ex2_approx(pwq[1]));
            float2 bank = f2(h1.w);
#pragma unroll
            for (int i = 0; i < K; ++i) {
              const float2 a = reduced_angle2<decltype(fast_tag)::value>(thp[i]);
              bank = __ffma2_rn(f2(fr[2 * K + i]), make_float2(__cosf(a.x), __cosf(a.y)), bank);
            }
            float2 al = __fmul2_rn(__fmul2_rn(f2(h1.z), G), bank);
            al.x = fminf(amax, al.x);
            al.y = fminf(amax, al.y);
            const float2 Tp = make_float2(T[0], T[1]);
            const float2 test = __fmul2_rn(Tp, __ffma2_rn(al, f2(-1.f), f2(1.f)));   // T (1 - alpha)
            float2 wgt = __fmul2_rn(al, Tp);
            const bool pass0 = reach[0] && al.x >= amin, pass1 = reach[1] && al.y >= amin;
            const bool stop0 = pass0 && test.x < Tmin, stop1 = pass1 && test.y < Tmin;
            const bool comp0 = pass0 && !stop0, comp1 = pass1 && !stop1;
            const u32 here = start + (u32)j + 1u - rg.x;
            if (STATS) {
              reached[0] += reach[0] ? 1u : 0u;
              reached[1] += reach[1] ? 1u : 0u;
              if (stop0) evaluated[0] = here;
              if (stop1) evaluated[1] = here;
              composited[0] += comp0 ? 1u : 0u;
              composited[1] += comp1 ? 1u : 0u;
            }
            if (stop0) done[0] = true;
            if (stop1) done[1] = true;
            if (comp0) { T[0] = test.x; last[0] = here; } else { wgt.x = 0.f; }
            if (comp1) { T[1] = test.y; last[1] = here; } else { wgt.y = 0.f; }
            const float4 c = r[2];   // a zero weight leaves the (non-negative) sums unchanged
            const float2 s0 = __ffma2_rn(f2(c.x), wgt, make_float2(C0[0], C0[1]));
            const float2 s1 = __ffma2_rn(f2(c.y), wgt, make_float2(C1[0], C1[1]));
            const float2 s2 = __ffma2_rn(f2(c.z), wgt, make_float2(C2[0], C2[1]));
            C0[0] = s0.x; C0[1] = s0.y;
            C1[0] = s1.x; C1[1] = s1.y;
            C2[0] = s2.x; C2[1] = s2.y;
            comp = comp0 || comp1;
          } else {
            float th[K > 0 ? K : 1];
#pragma unroll
            for (int i = 0; i < K; ++i) th[i] = raw_phase(fr[2 * i], fr[2 * i + 1], dx, dyq[0]);
#pragma unroll
            for (int q = 0; q < PPT; ++q) {
              if (q > 0)
#pragma unroll
                for (int i = 0; i < K; ++i) th[i] = __fadd_rn(th[i], fr[2 * i + 1]);
              if (reach[q]) {
                if (STATS) ++reached[q];
                const float G = ex2_approx(pwq[q]);
                const float bank = filter_bank<K, decltype(fast_tag)::value>(th, fr + 2 * K, h1.w);
                const float alpha = fminf(amax, __fmul_rn(__fmul_rn(h1.z, G), bank));
                if (alpha >= amin) {
                  const float test = __fmul_rn(T[q], __fsub_rn(1.f, alpha));
                  if (test < Tmin) {
                    done[q] = true;
                    if (STATS) evaluated[q] = start + (u32)j + 1u - rg.x;
                  } else {
                    const float4 c = r[2];
                    const float wgt = alpha * T[q];
                    C0[q] = __fmaf_rn(c.x, wgt, C0[q]);
                    C1[q] = __fmaf_rn(c.y, wgt, C1[q]);
                    C2[q] = __fmaf_rn(c.z, wgt, C2[q]);
                    T[q] = test;
                    last[q] = start + (u32)j + 1u - rg.x;
                    if (STATS) ++composited[q];
                    comp = true;
                  }
                }
              }
            }
          }
        };
        // with the composited-pair bits every lane walks the whole word, so the branch can be a
        // warp vote: the lanes without a reached pixel run the same instructions and keep nothing
        if (MASKS ? __any_sync(0xffffffffu, any) : any) {
          if (fast)
            pixels(std::true_type{});
          else
            pixels(std::false_type{});
        }
        tdone = true;
#pragma unroll
        for (int q = 0; q < PPT; ++q) tdone = tdone && done[q];
        if (MASKS && comp) lbits |= 1u << ((start + (u32)j) & 31u);
      }
      if (MASKS) {
        const u32 cw = __reduce_or_sync(0xffffffffu, lbits);
        if (lane == 0) cplane[(start >> 5) + tile] = cw;
      }
      __syncwarp();   // every lane is done with the staged rows before the next word is staged
      start = end;
    }
    float* orgb = out_rgb ? out_rgb : V.out_rgb;
    float* oT = out_rgb ? out_T : V.out_T;
    const size_t hw = (size_t)V.width * V.height;
#pragma unroll
    for (int q = 0; q < PPT; ++q) {
      const int py = py0 + q;
      if (px < V.width && py < V.height) {
        const size_t pix = (size_t)py * V.width + px;
        if (orgb) {
          orgb[pix] = FMAP ? C0[q] : C0[q] + T[q] * tbl->bg[0];
          orgb[hw + pix] = FMAP ? C1[q] : C1[q] + T[q] * tbl->bg[1];
          orgb[2 * hw + pix] = FMAP ? C2[q] : C2[q] + T[q] * tbl->bg[2];
        }
        if (oT) oT[pix] = T[q];
        p.T_final[V.pix_base + pix] = T[q];
        p.n_contrib[V.pix_base + pix] = last[q];
        if (STATS) {
          p.n_eval[V.pix_base + pix] = evaluated[q];
          p.n_reach[V.pix_base + pix] = reached[q];
          p.n_comp[V.pix_base + pix] = composited[q];
        }
      }
    }
  }
  __syncthreads();   // every warp of the CTA has left its task loop
  if (threadIdx.x == 0) release_tile_counter(&hdr->tile_counter_fwd, &hdr->fwd_exits);
}

// Per-thread pixel state of the reverse walk (PPT vertically adjacent pixels).
template <int PPT>
struct BwdPix {
  // tbg: T_final (bg . dL/dC), the background's share of dL/dalpha (scaled by 1 / (1 - alpha))
  float T[PPT], g0[PPT], g1[PPT], g2[PPT], tbg[PPT], acc0[PPT], acc1[PPT], acc2[PPT];
  u32 last[PPT];
};

// One pair's adjoint at a thread's PPT pixels (Eq. 9-10 differentiated, back to front): restores
// the transmittance before the pair, updates the colour sums behind it and adds the pair's
// gradient contributions into col, its column of the warp's transpose buffer.  pos: 0-based position of the pair in the
// tile list.  Returns whether a pixel of the thread composited the pair.  The envelope, bank and
// alpha are evaluated exactly as the forward evaluates them, so both take the same decisions.
// Row stride (floats) of a warp's transpose buffer: value v of lane l at [v * BWD_RS + l]; 36 keeps
// the reading lanes' 16-byte loads free of bank conflicts.
constexpr int BWD_RS = 36;

template <int K, int PPT, bool FAST>
__device__ __forceinline__ bool pair_adjoint(BwdPix<PPT>& S, const float4* r, u32 pos, float fpx, float fpy0,
                                             float amin, float amax, float* col) {
  constexpr int NV = 10 + 3 * K;
  const float4 h0 = r[0], h1 = r[1];
  const float* fw = reinterpret_cast<const float*>(r + 3);   // 2 pi f2D, then the weights
  const float dx = __fsub_rn(fpx, h0.x);
  const float oln2 = h1.z * 0.6931471805599453f;   // opacity ln 2
  bool contrib = false;
  float dyq[PPT], pwq[PPT];
  pixel_powers<PPT>(h0, h1, dx, __fsub_rn(fpy0, h0.y), dyq, pwq);
  if constexpr (PPT == 2 && K <= GS_BWD_PACKED_MAX_K) {
    // Both pixels at once.  Envelope, bank and alpha in packed FP32, bit-identical to the
    // forward's decisions.  A pixel that does not take part gets alpha 0 (its transmittance
    // and colour sums stay as they are) and dL/dalpha 0 (it adds exact zeros), and the two
    // pixels' adjoints are summed before they meet the shared factors: dx is common, and
    // sums against dy use each pixel's own offset.  The code is straight-line: a pair is
    // walked only where a pixel of the warp composited it, so a lane leaving early would
    // only wait, and its column stores would no longer coincide with the other lanes'.
    const bool live0 = pos < S.last[0] && pwq[0] >= h1.y;
    const bool live1 = pos < S.last[1] && pwq[1] >= h1.y;
    float2 thp[K > 0 ? K : 1];
#pragma unroll
    for (int i = 0; i < K; ++i) thp[i] = row_phases2(fw[2 * i], fw[2 * i + 1], dx, dyq);
    const float2 G = make_float2(ex2_approx(pwq[0]), ex2_approx(pwq[1]));
    float2 cs[K > 0 ? K : 1], sn[K > 0 ? K : 1];
    float2 bank = f2(h1.w);
#pragma unroll
    for (int i = 0; i < K; ++i) {
      const float2 a = reduced_angle2<FAST>(thp[i]);
      cs[i] = make_float2(__cosf(a.x), __cosf(a.y));
      sn[i] = make_float2(__sinf(a.x), __sinf(a.y));
      bank = __ffma2_rn(f2(fw[2 * K + i]), cs[i], bank);
    }
    const float2 araw = __fmul2_rn(__fmul2_rn(f2(h1.z), G), bank);
    const float ax = fminf(amax, araw.x), ay = fminf(amax, araw.y);
    const bool pass0 = live0 && ax >= amin, pass1 = live1 && ay >= amin;
    contrib = pass0 || pass1;
    const float2 alpha = make_float2(pass0 ? ax : 0.f, pass1 ? ay : 0.f);
    const float2 oma = __ffma2_rn(alpha, f2(-1.f), f2(1.f));
    const float2 ioma = make_float2(rcp_approx(oma.x), rcp_approx(oma.y));
    const float2 Tn = __fmul2_rn(make_float2(S.T[0], S.T[1]), ioma);   // transmittance before this pair
    if (pass0) S.T[0] = Tn.x;
    if (pass1) S.T[1] = Tn.y;
    const float4 c = r[2];
    const float2 wgt = __fmul2_rn(alpha, Tn);
    const float2 G0 = make_float2(S.g0[0], S.g0[1]), G1 = make_float2(S.g1[0], S.g1[1]), G2 = make_float2(S.g2[0], S.g2[1]);
    float2 A0 = make_float2(S.acc0[0], S.acc0[1]), A1 = make_float2(S.acc1[0], S.acc1[1]),
           A2 = make_float2(S.acc2[0], S.acc2[1]);
    // (c - acc) . dL/dC, then dL/dalpha = T (c - acc) . dL/dC - tbg / (1 - alpha)
    float2 dcg = __fmul2_rn(__ffma2_rn(A2, f2(-1.f), f2(c.z)), G2);
    dcg = __ffma2_rn(__ffma2_rn(A1, f2(-1.f), f2(c.y)), G1, dcg);
    dcg = __ffma2_rn(__ffma2_rn(A0, f2(-1.f), f2(c.x)), G0, dcg);
    float2 dLda = __ffma2_rn(__fmul2_rn(make_float2(S.tbg[0], S.tbg[1]), ioma), f2(-1.f), __fmul2_rn(Tn, dcg));
    A0 = __ffma2_rn(oma, A0, __fmul2_rn(alpha, f2(c.x)));
    A1 = __ffma2_rn(oma, A1, __fmul2_rn(alpha, f2(c.y)));
    A2 = __ffma2_rn(oma, A2, __fmul2_rn(alpha, f2(c.z)));
    S.acc0[0] = A0.x; S.acc0[1] = A0.y;
    S.acc1[0] = A1.x; S.acc1[1] = A1.y;
    S.acc2[0] = A2.x; S.acc2[1] = A2.y;
    // no gradient through a clamped alpha, none from a pixel that does not take part
    if (!pass0 || araw.x > amax) dLda.x = 0.f;
    if (!pass1 || araw.y > amax) dLda.y = 0.f;
    col[(6) * BWD_RS] = fmaf(wgt.y, S.g0[1], wgt.x * S.g0[0]);
    col[(7) * BWD_RS] = fmaf(wgt.y, S.g1[1], wgt.x * S.g1[0]);
    col[(8) * BWD_RS] = fmaf(wgt.y, S.g2[1], wgt.x * S.g2[0]);
    const float2 dLdG = __fmul2_rn(dLda, G);
    const float2 dLdbank = __fmul2_rn(dLdG, f2(h1.z));
    const float2 dLdo = __fmul2_rn(dLdG, bank);
    // log2-domain power p2: G = 2^p2, dG/dp2 = G ln 2, so dL/dp2 = dLda o bank G ln 2
    const float2 dLdp2 = __fmul2_rn(dLdo, f2(oln2));
    const float2 edy = __fmul2_rn(dLdp2, make_float2(dyq[0], dyq[1]));
    const float P = dLdp2.x + dLdp2.y;               // sum of dL/dp2
    const float Y = edy.x + edy.y;                   // sum of dL/dp2 dy
    const float Ex = P * dx;                         // sum of dL/dp2 dx
    col[(5) * BWD_RS] = dLdo.x + dLdo.y;                         // d opacity
    col[(2) * BWD_RS] = Ex * dx;                                 // w.r.t. A' (converted at flush)
    col[(3) * BWD_RS] = Y * dx;                                  // w.r.t. B'
    col[(4) * BWD_RS] = fmaf(edy.y, dyq[1], edy.x * dyq[0]);     // w.r.t. C'
    float gdx = 2.f * h0.z * Ex + h0.w * Y;
    float gdy = h0.w * Ex + 2.f * h1.x * Y;
#pragma unroll
    for (int i = 0; i < K; ++i) {
      const float wi = fw[2 * K + i];
      const float2 kc = __fmul2_rn(dLdbank, cs[i]);
      const float2 ks = __fmul2_rn(dLdbank, sn[i]);
      col[(9 + 2 * K + i) * BWD_RS] = kc.x + kc.y;                         // d (cosine weight i)
      const float gth = -wi * (ks.x + ks.y);                   // d phase (radians), both pixels
      const float gthdy = -wi * fmaf(ks.y, dyq[1], ks.x * dyq[0]);
      col[(9 + 2 * i) * BWD_RS] = gth * dx;                                // w.r.t. 2 pi f2D (scaled at flush)
      col[(9 + 2 * i + 1) * BWD_RS] = gthdy;
      gdx += gth * fw[2 * i];
      gdy += gth * fw[2 * i + 1];
    }
    col[(9 + 3 * K) * BWD_RS] = dLdbank.x + dLdbank.y;           // d (1 - sum w)
    col[(0) * BWD_RS] = -gdx;                                    // d mu = - d (pixel - mu)
    col[(1) * BWD_RS] = -gdy;
  } else {
    float gv[NV];
#pragma unroll
    for (int i = 0; i < NV; ++i) gv[i] = 0.f;
    // raw phases of the current row, taken as the forward takes them (two rows: row_phases2)
    float th[K > 0 ? K : 1], th1[K > 0 ? K : 1];
#pragma unroll
    for (int i = 0; i < K; ++i) {
      if constexpr (PPT == 2) {
        const float2 t = row_phases2(fw[2 * i], fw[2 * i + 1], dx, dyq);
        th[i] = t.x;
        th1[i] = t.y;
      } else {
        th[i] = raw_phase(fw[2 * i], fw[2 * i + 1], dx, dyq[0]);
      }
    }
#pragma unroll
    for (int q = 0; q < PPT; ++q) {
      if (q > 0)
#pragma unroll
        for (int i = 0; i < K; ++i) th[i] = PPT == 2 ? th1[i] : __fadd_rn(th[i], fw[2 * i + 1]);
      if (pos >= S.last[q]) continue;
      const float dy = dyq[q];
      const float pw = pwq[q];
      if (pw < h1.y) continue;
      const float G = ex2_approx(pw);
      float cs[K > 0 ? K : 1], sn[K > 0 ? K : 1];
      float bank = h1.w;
#pragma unroll
      for (int i = 0; i < K; ++i) {
        const float ang = reduced_angle<FAST>(th[i]);
        cs[i] = __cosf(ang);
        sn[i] = __sinf(ang);
      }
#pragma unroll
      for (int i = 0; i < K; ++i) bank = __fmaf_rn(fw[2 * K + i], cs[i], bank);
      const float araw = __fmul_rn(__fmul_rn(h1.z, G), bank);
      const float alpha = fminf(amax, araw);
      if (alpha < amin) continue;
      contrib = true;
      const float oma = 1.f - alpha;
      const float ioma = rcp_approx(oma);
      S.T[q] = S.T[q] * ioma;                              // transmittance before this pair
      const float4 c = r[2];
      const float wgt = alpha * S.T[q];
      gv[6] += wgt * S.g0[q];
      gv[7] += wgt * S.g1[q];
      gv[8] += wgt * S.g2[q];
      float dLda = S.T[q] * ((c.x - S.acc0[q]) * S.g0[q] + (c.y - S.acc1[q]) * S.g1[q] + (c.z - S.acc2[q]) * S.g2[q]) -
                   S.tbg[q] * ioma;
      S.acc0[q] = alpha * c.x + oma * S.acc0[q];
      S.acc1[q] = alpha * c.y + oma * S.acc1[q];
      S.acc2[q] = alpha * c.z + oma * S.acc2[q];
      if (araw > amax) dLda = 0.f;                     // clamped: no gradient through alpha
      const float dLdG = dLda * G;
      const float dLdbank = dLdG * h1.z;
      const float dLdo = dLdG * bank;
      gv[5] += dLdo;                                   // d opacity
      // log2-domain power p2: G = 2^p2, dG/dp2 = G ln 2, so dL/dp2 = dLda o bank G ln 2
      const float dLdp2 = dLdo * oln2;
      const float ex = dLdp2 * dx, ey = dLdp2 * dy;
      gv[2] += ex * dx;                                // w.r.t. A' (converted at flush)
      gv[3] += ex * dy;                                // w.r.t. B'
      gv[4] += ey * dy;                                // w.r.t. C'
      float gdx = 2.f * h0.z * ex + h0.w * ey;
      float gdy = h0.w * ex + 2.f * h1.x * ey;
#pragma unroll
      for (int i = 0; i < K; ++i) {
        const float wi = fw[2 * K + i];
        gv[9 + 2 * K + i] += dLdbank * cs[i];                  // d (cosine weight i)
        const float gth = -dLdbank * wi * sn[i];                // d phase (radians)
        gv[9 + 2 * i] += gth * dx;                              // w.r.t. 2 pi f2D (scaled at flush)
        gv[9 + 2 * i + 1] += gth * dy;
        gdx += gth * fw[2 * i];
        gdy += gth * fw[2 * i + 1];
      }
      gv[9 + 3 * K] += dLdbank;                        // d (1 - sum w)
      gv[0] -= gdx;                                    // d mu = - d (pixel - mu)
      gv[1] -= gdy;
    }
#pragma unroll
    for (int i = 0; i < NV; ++i) col[i * BWD_RS] = gv[i];
  }
  return contrib;
}
// Chunks [c0, c0 + count) of a zero-fill, by one warp (zero_chunks with lane strides).
__device__ __noinline__ void zero_chunks_warp(const ZeroJob& z, u32 c0, u32 count, int lane) {
  const u32 total = z.base[ZERO_ARRAYS];
  const u32 c1 = c0 < total - min(total, count) ? c0 + count : total;
  for (u32 c = c0; c < c1; ++c) {
    int i = 0;
    while (c >= z.base[i + 1]) ++i;   // c < total: ends at an array that owns chunk c
    const u64 off = (u64)(c - z.base[i]) * ZERO_CHUNK;
    const u32 len = (u32)min((u64)ZERO_CHUNK, z.n[i] - off);
    float* a = z.a[i] + off;
    u32 done = 0;
    if ((reinterpret_cast<uintptr_t>(z.a[i]) & 15u) == 0) {
      const u32 n4 = len >> 2;
      for (u32 j = (u32)lane; j < n4; j += 32u) __stcs(reinterpret_cast<float4*>(a) + j, make_float4(0.f, 0.f, 0.f, 0.f));
      done = 4 * n4;
    }
    for (u32 j = done + (u32)lane; j < len; j += 32u) a[j] = 0.f;
  }
}

// Position of the (r + 1)-th highest set bit of m (m has more than r set bits): the largest b with
// popc(m >> b) > r.
__device__ __forceinline__ int nth_high_bit(u32 m, int r) {
  int b = 0;
#pragma unroll
  for (int s = 16; s; s >>= 1)
    if (__popc(m >> (b + s)) > r) b += s;
  return b;
}

// Warps of one tile: one per 8x8 (PPT = 2) footprint, the units the forward records
// composited-pair bits for.
constexpr int BWD_WARPS_PER_TILE = BLOCK / GS_PPT_BWD / 32;

// The reverse walk with independent warps.  A task is one warp footprint of one tile (tiles in the
// order of tile_order, longest pair lists first); a warp takes tasks from the device counter, walks
// the pairs that the forward recorded as composited by its pixels, back to front, staging them 32
// at a time into its own shared-memory rows, and adds each pair's warp-reduced gradients straight
// into the pair's grad2d row with vector reductions.  No CTA barrier sits on the walk, so a warp
// with little work moves on instead of waiting for the others of its CTA.  After each task the
// warp zero-fills its share of the attribute gradients.
template <int K, int PPT>
__global__ void GS_BWD_BOUNDS k_render_bwd_w(WsPtrs p, const float* __restrict__ dL_drgb,
                                             const __grid_constant__ ZeroJob z) {
  pdl_begin();
  constexpr int NW = BLOCK / PPT / 32;   // warps per CTA
  constexpr int WPT = BWD_WARPS_PER_TILE;
  constexpr int F4 = SRec<K>::F4;
  constexpr int NV = 10 + 3 * K;         // gradient values per pair
  constexpr int NG = g2d_floats(K);      // padded row in global memory
  constexpr int NVP = (NV + 31) / 32 * 32;
  // the packed adjoint's unroll (K > 4: its own factor); the per-pixel adjoint: no unroll
  constexpr int BWD_UNR = K <= 4 ? BWD_UNROLL : K <= GS_BWD_PACKED_MAX_K ? GS_BWD_UNROLL_HIGHK : 1;
  extern __shared__ __align__(16) float4 smem4[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float4* s_rec = smem4 + warp * 32 * F4;                                              // [32][F4]
  u32* s_id = reinterpret_cast<u32*>(smem4 + NW * 32 * F4) + warp * 64;                // [32] rows
  u32* s_pos = s_id + 32;                                                              // [32] positions
  float* s_red = reinterpret_cast<float*>(smem4 + NW * 32 * F4 + NW * 16) + warp * (NV * BWD_RS + 4);
  WsHeader* hdr = p.hdr;
  if (read_status(hdr) != 0) return;
  if (hdr->masks_epoch != hdr->epoch) {   // no forward of this frame recorded the composited-pair bits
    if (blockIdx.x == 0 && threadIdx.x == 0) set_status(hdr, GS_ERR_INVALID_ARG);
    return;
  }
  const FrameTable* tbl = p.tbl;
  // sorted pairs tile << 32 | depth rank; the rank is the record (and grad2d) row
  const u64* __restrict__ pairs = (tbl->tpasses_needed & 1) ? p.keys1 : p.keys0;
  const u32 ntiles = tbl->total_tiles;
  const float amax = tbl->alpha_max, amin = tbl->alpha_min;
  // lane v's share of the record-gradient conversion: log2-domain conic (A' = -a/2 log2 e,
  // B' = -b log2 e, C' = -c/2 log2 e) to (a, b, c), and the staged 2 pi f2D to f2D
  float conv[NVP / 32];
#pragma unroll
  for (int g = 0; g < NVP / 32; ++g) {
    const int v = 32 * g + lane;
    conv[g] = (v == 2 || v == 4) ? -0.5f * LOG2E : v == 3 ? -LOG2E : (v >= 9 && v < 9 + 2 * K) ? TWO_PI : 1.f;
  }
  for (;;) {
    u32 slot = 0;
    if (lane == 0) slot = atomicAdd(&hdr->tile_counter_bwd, 1u);
    slot = __shfl_sync(0xffffffffu, slot, 0);
    if (slot >= ntiles * (u32)WPT) break;   // warp-uniform
    const u32 tile = p.tile_order[slot / WPT];
    const int quad = (int)(slot % WPT);
    const int v = view_of_tile(tbl, tile);
    const ViewDesc& V = tbl->v[v];
    const u32 local = tile - V.tile_base;
    const int tx = (int)(local % (u32)V.tiles_x), ty = (int)(local / (u32)V.tiles_x);
    const int2 pxy = thread_pixel<PPT>(tx, ty, quad * 32 + lane);
    const int px = pxy.x, py0 = pxy.y;
    const uint2 rg = p.ranges[tile];
    const float fpx = (float)px + 0.5f, fpy0 = (float)py0 + 0.5f;
    const float* gsrc = dL_drgb ? dL_drgb : V.dL_drgb;
    const size_t hw = (size_t)V.width * V.height;
    BwdPix<PPT> S;
    u32 wlast = 0;
#pragma unroll
    for (int q = 0; q < PPT; ++q) {
      S.T[q] = 1.f;
      S.g0[q] = S.g1[q] = S.g2[q] = 0.f;
      S.acc0[q] = S.acc1[q] = S.acc2[q] = 0.f;
      S.last[q] = 0;
      const int py = py0 + q;
      if (px < V.width && py < V.height) {
        const size_t pix = (size_t)py * V.width + px;
        S.T[q] = p.T_final[V.pix_base + pix];
        S.last[q] = p.n_contrib[V.pix_base + pix];
        S.g0[q] = gsrc[pix];
        S.g1[q] = gsrc[hw + pix];
        S.g2[q] = gsrc[2 * hw + pix];
      }
      S.tbg[q] = S.T[q] * (tbl->bg[0] * S.g0[q] + tbl->bg[1] * S.g1[q] + tbl->bg[2] * S.g2[q]);
      wlast = max(wlast, S.last[q]);
    }
    // the last composited pair over the warp bounds the reverse walk: sorted positions [rg.x, hi)
#pragma unroll
    for (int o = 16; o; o >>= 1) wlast = max(wlast, __shfl_xor_sync(0xffffffffu, wlast, o));
    const u32 lo = rg.x, hi = rg.x + wlast;
    const u32* cplane = p.cmask + (size_t)quad * p.cmask_plane;
    const int wk_bot = (int)(lo >> 5);
    int wk_top = hi > lo ? (int)((hi - 1) >> 5) : wk_bot - 1;   // highest word still to walk
    while (wk_top >= wk_bot) {   // warp-uniform
      // collect: lane l reads word wk_top - l; the leading words whose bits add up to at most 32
      // are taken, and lane s finds the s-th highest of their set bits
      const int wk = wk_top - lane;
      u32 m = 0;
      if (wk >= wk_bot) {
        const u32 w0 = (u32)wk << 5;
        m = cplane[(u32)wk + tile];
        if (w0 < lo) m &= ~0u << (lo - w0);
        if (hi - w0 < 32u) m &= (1u << (hi - w0)) - 1u;
      }
      const int c = __popc(m);
      int incl = c;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
      }
      const int excl = incl - c;
      const int nw = __popc(__ballot_sync(0xffffffffu, incl <= 32 && wk >= wk_bot));   // >= 1
      const int total = __shfl_sync(0xffffffffu, incl, nw - 1);
      int j = 0;   // the word holding slot `lane`: the largest j < nw with excl_j <= lane
#pragma unroll
      for (int s = 16; s; s >>= 1) {
        const int e = __shfl_sync(0xffffffffu, excl, (j + s) & 31);
        if (j + s < nw && e <= lane) j += s;
      }
      const u32 mj = __shfl_sync(0xffffffffu, m, j);
      const int ej = __shfl_sync(0xffffffffu, excl, j);
      if (lane < total) {
        const u32 pos = ((u32)(wk_top - j) << 5) + (u32)nth_high_bit(mj, lane - ej);
        const u32 id = (u32)pairs[pos];
        s_id[lane] = id;
        s_pos[lane] = pos - lo;   // 0-based position in the tile list
        float2 flo, fhi;
        footprint_bounds<PPT>(fpx, fpy0, lane, flo, fhi);
        stage_record<K>(p.records + (size_t)id * rec_floats(K), s_rec + lane * F4, amin, flo, fhi);
      }
      wk_top -= nw;
      __syncwarp();
#pragma unroll BWD_UNR
      for (int sl = 0; sl < total; ++sl) {   // descending positions
        const float4* r = s_rec + sl * F4;
        const bool fast = reinterpret_cast<const float*>(r)[11] != 0.f;   // the same for every lane
        const u32 pos = s_pos[sl];
        // every walked pair was composited by a pixel of the warp: each lane stores its gradient
        // values in its column of the transpose buffer (value v in row v), lane v adds up row v
        // with eight 16-byte loads, and lanes 4i add values 4i .. 4i + 3 to the pair's grad2d row
        // with one vector reduction
        if (fast)
          pair_adjoint<K, PPT, true>(S, r, pos, fpx, fpy0, amin, amax, s_red + lane);
        else
          pair_adjoint<K, PPT, false>(S, r, pos, fpx, fpy0, amin, amax, s_red + lane);
        {
          __syncwarp();
          float* dst = p.grad2d + (size_t)s_id[sl] * NG;
#pragma unroll
          for (int g = 0; g < NVP / 32; ++g) {
            const int vv = 32 * g + lane;
            float sum = 0.f;
            if (vv < NV) {
              const float4* row = reinterpret_cast<const float4*>(s_red + vv * BWD_RS);
              const float4 a = row[0];
              float2 l2 = make_float2(a.x, a.y), h2 = make_float2(a.z, a.w);   // packed column sums
#pragma unroll
              for (int cc = 1; cc < 8; ++cc) {
                const float4 t = row[cc];
                l2 = __fadd2_rn(l2, make_float2(t.x, t.y));
                h2 = __fadd2_rn(h2, make_float2(t.z, t.w));
              }
              sum = ((l2.x + l2.y) + (h2.x + h2.y)) * conv[g];
            }
            const float s1 = __shfl_down_sync(0xffffffffu, sum, 1);
            const float s2 = __shfl_down_sync(0xffffffffu, sum, 2);
            const float s3 = __shfl_down_sync(0xffffffffu, sum, 3);
            if ((lane & 3) == 0 && vv < NG && (sum != 0.f || s1 != 0.f || s2 != 0.f || s3 != 0.f))
              asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(dst + vv), "f"(sum), "f"(s1),
                           "f"(s2), "f"(s3)
                           : "memory");
          }
          __syncwarp();
        }
      }
      __syncwarp();   // every lane is done with the staged rows before the next collection
    }
    if (z.quota) {   // this task's share of the zero-fill, issued behind its walk
      u32 c0 = 0;
      if (lane == 0) c0 = atomicAdd(&hdr->zero_counter, z.quota);
      zero_chunks_warp(z, __shfl_sync(0xffffffffu, c0, 0), z.quota, lane);
    }
  }
  // the task queue is empty: the chunks still unclaimed
  if (z.quota) {
    for (;;) {
      u32 c0 = 0;
      if (lane == 0) c0 = atomicAdd(&hdr->zero_counter, z.quota);
      c0 = __shfl_sync(0xffffffffu, c0, 0);
      if (c0 >= z.base[ZERO_ARRAYS]) break;   // warp-uniform
      zero_chunks_warp(z, c0, z.quota, lane);
    }
  }
  __syncthreads();   // every warp of the CTA has left its task loop
  if (threadIdx.x == 0) release_tile_counter(&hdr->tile_counter_bwd, &hdr->bwd_exits, &hdr->zero_counter);
}

template <int K, bool FMAP, bool MASKS, bool STATS>
static cudaError_t launch_fwd_t(const FrameTable& tbl, const WsPtrs& p, float* rgb, float* T,
                                const Launch& L) {
  constexpr int PPT = GS_PPT_FWD, NT = BLOCK / PPT;
  static int grid = 0;
  const size_t smem = (size_t)NT * SRec<K>::F * sizeof(float);   // 32 rows per warp
  auto kern = k_render_fwd_w<K, PPT, FMAP, MASKS, STATS>;
  if (!grid) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NT, smem) != cudaSuccess || per_sm < 1) per_sm = 1;
    grid = per_sm * L.sm_count;
  }
  int g = grid;
  if ((u32)g > tbl.launch_tiles) g = (int)tbl.launch_tiles;   // one task per warp footprint: NT / 32 per tile
  if (g < 1) g = 1;
  launch_pdl<PDL_RENDER>(kern, g, NT, smem, L.stream, p, rgb, T);
  return cudaGetLastError();
}

// Clears the 2D gradient rows of the n_active ranked primitives before the backward accumulates.
template <int K>
__global__ void __launch_bounds__(256) k_zero_grad2d(WsPtrs p) {
  pdl_begin();
  if (read_status(p.hdr) != 0) return;
  static_assert(g2d_floats(K) % 4 == 0, "grad2d rows are whole float4s");
  const size_t n4 = (size_t)p.hdr->n_active * (g2d_floats(K) / 4);
  float4* g = reinterpret_cast<float4*>(p.grad2d);
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += (size_t)gridDim.x * blockDim.x)
    g[i] = make_float4(0.f, 0.f, 0.f, 0.f);
}

template <int K>
static cudaError_t launch_bwd_t(const FrameTable& tbl, const WsPtrs& p, const float* dL, const ZeroJob* z,
                                const Launch& L) {
  constexpr int PPT = GS_PPT_BWD, NT = BLOCK / PPT;
  static int grid = 0;
  constexpr int NW = NT / 32;
  const size_t smem = (size_t)NW * (32 * SRec<K>::F * sizeof(float) + 64 * sizeof(u32) +
                                    ((10 + 3 * K) * 36 + 4) * sizeof(float));
  if (!grid) {
    cudaError_t e =
        cudaFuncSetAttribute(k_render_bwd_w<K, PPT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_render_bwd_w<K, PPT>, NT, smem) != cudaSuccess ||
        per_sm < 1)
      per_sm = 1;
    grid = per_sm * L.sm_count;
  }
  int g = grid;
  if ((u32)g > tbl.launch_tiles) g = (int)tbl.launch_tiles;   // one task per warp footprint: NW per tile
  if (g < 1) g = 1;
  ZeroJob zw{};
  if (z) {   // the fill's chunks per tile spread over the tile's warp tasks
    zw = *z;
    if (zw.quota) zw.quota = (zw.quota + BWD_WARPS_PER_TILE - 1) / BWD_WARPS_PER_TILE;
  }
  launch_pdl<PDL_RENDER>(k_zero_grad2d<K>, L.sm_count * 2, 256, 0, L.stream, p);
  launch_pdl<PDL_RENDER>(k_render_bwd_w<K, PPT>, g, NT, smem, L.stream, p, dL, zw);
  return cudaGetLastError();
}


template <bool FMAP, bool MASKS, bool STATS>
static cudaError_t launch_fwd_k(const FrameTable& tbl, const WsPtrs& p, float* out, float* out_T, const Launch& L) {
  switch (tbl.K) {
    case 0: return launch_fwd_t<0, FMAP, MASKS, STATS>(tbl, p, out, out_T, L);
    case 1: return launch_fwd_t<1, FMAP, MASKS, STATS>(tbl, p, out, out_T, L);
    case 2: return launch_fwd_t<2, FMAP, MASKS, STATS>(tbl, p, out, out_T, L);
    case 3: return launch_fwd_t<3, FMAP, MASKS, STATS>(tbl, p, out, out_T, L);
    case 4: return launch_fwd_t<4, FMAP, MASKS, STATS>(tbl, p, out, out_T, L);
    case 5: return launch_fwd_t<5, FMAP, MASKS, STATS>(tbl, p, out, out_T, L);
    case 6: return launch_fwd_t<6, FMAP, MASKS, STATS>(tbl, p, out, out_T, L);
    case 7: return launch_fwd_t<7, FMAP, MASKS, STATS>(tbl, p, out, out_T, L);
    case 8: return launch_fwd_t<8, FMAP, MASKS, STATS>(tbl, p, out, out_T, L);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_render_fwd(const FrameTable& tbl, const WsPtrs& p, float* out_rgb, float* out_T, const Launch& L,
                              bool masks, bool stats) {
  if (!masks) return launch_fwd_k<false, false, false>(tbl, p, out_rgb, out_T, L);
  return stats ? launch_fwd_k<false, true, true>(tbl, p, out_rgb, out_T, L)
               : launch_fwd_k<false, true, false>(tbl, p, out_rgb, out_T, L);
}

cudaError_t launch_render_freq_map(const FrameTable& tbl, const WsPtrs& p, float* out_map, const Launch& L) {
  return launch_fwd_k<true, false, false>(tbl, p, out_map, nullptr, L);
}

cudaError_t launch_render_bwd(const FrameTable& tbl, const WsPtrs& p, const float* dL, const ZeroJob* z,
                              const Launch& L) {
  switch (tbl.K) {
    case 0: return launch_bwd_t<0>(tbl, p, dL, z, L);
    case 1: return launch_bwd_t<1>(tbl, p, dL, z, L);
    case 2: return launch_bwd_t<2>(tbl, p, dL, z, L);
    case 3: return launch_bwd_t<3>(tbl, p, dL, z, L);
    case 4: return launch_bwd_t<4>(tbl, p, dL, z, L);
    case 5: return launch_bwd_t<5>(tbl, p, dL, z, L);
    case 6: return launch_bwd_t<6>(tbl, p, dL, z, L);
    case 7: return launch_bwd_t<7>(tbl, p, dL, z, L);
    case 8: return launch_bwd_t<8>(tbl, p, dL, z, L);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace gs
