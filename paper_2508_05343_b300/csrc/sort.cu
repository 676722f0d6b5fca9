// Depth ordering of the (tile, primitive) pairs (Sec. 3.1 "sorted by depth", Sec. 3.3.3 tile
// rasterizer) in two stable least-significant-digit radix sorts of 64-bit keys, each digit pass one
// "onesweep" kernel: a CTA ranks its partition locally, obtains the global offset of every digit by
// decoupled look-back over the preceding partitions, and scatters through shared memory so global
// writes are coalesced.
//   1. Depth sort of the active primitives (in the preprocess stage): keys
//      (float bits of depth - bits of znear) << 32 | primitive, over the depth_bits significant bits.
//      Positive floats order like their bit patterns; the input is in primitive order, so equal
//      depths keep primitive order.  The position of a primitive in the result is its depth rank.
//   2. Tile sort of the pairs (this stage): the emission writes tile << 32 | depth rank in rank
//      order, so a stable sort on the tile bits alone leaves every tile's pairs in depth order
//      (ties by primitive index): the order of a sort of (tile, depth, primitive).
// Both sorts move 8-byte keys only.  Digit counts come from the active-list scan (depth) and from
// the emission (tile); counts stay on the device; persistent CTAs take partitions in order from an
// atomic counter.  The last depth pass also adds each rank chunk's kept-tile counts (the partials
// of the rank-order scan), and the last tile pass writes each tile's [start, end) range.
#include "common.cuh"

namespace gs {

static_assert(SORT_THREADS >= RADIX && SORT_THREADS % 32 == 0, "one digit per thread of the first RADIX threads");

// Ranking of a warp's keys by digit: 1 = the lanes sharing a digit from one vote per digit bit and
// the warp's digit counter bumped with one shared atomic; 0 = __match_any_sync and a shared
// read-modify-write of the counter.
#ifndef GS_SORT_BALLOT_RANK
#define GS_SORT_BALLOT_RANK 1
#endif

template <int ITEMS>
struct SortSmem {
  u32 warp_cnt[SORT_THREADS / 32][RADIX];
  u32 local_excl[RADIX];
  u32 glob[RADIX];
  u32 hist_excl[RADIX];
  u32 scratch[SORT_THREADS / 32];
  u32 part;
  u64 keys[SORT_THREADS * ITEMS];
};

// Exclusive scan of one value per thread over the CTA (two barriers); threads >= RADIX pass 0.
__device__ __forceinline__ u32 block_excl_scan(u32 v, u32* scratch /*SORT_THREADS / 32*/) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  u32 incl = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const u32 t = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += t;
  }
  if (lane == 31) scratch[warp] = incl;
  __syncthreads();
  u32 wbase = 0;
#pragma unroll
  for (int w = 0; w < SORT_THREADS / 32; ++w)
    if (w < warp) wbase += scratch[w];
  __syncthreads();
  return wbase + incl - v;
}

// One digit pass over bits [32 + 8 pass, 40 + 8 pass) of the keys, in partitions of
// SORT_THREADS * ITEMS keys.  slot < DPASSES: depth sort of the n_active primitive keys
// (pass = slot); otherwise tile sort of the pairs (pass = slot - DPASSES).
template <int ITEMS>
__global__ void __launch_bounds__(SORT_THREADS, GS_SORT_MIN_CTAS) k_onesweep(WsPtrs p, const u64* __restrict__ kin,
                                                                           u64* __restrict__ kout, int slot) {
  pdl_begin();
  constexpr int PART = SORT_THREADS * ITEMS;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  SortSmem<ITEMS>& S = *reinterpret_cast<SortSmem<ITEMS>*>(smem_raw);
  WsHeader* hdr = p.hdr;
  if (read_status(hdr) != 0) return;
  const bool tiles = slot >= DPASSES;
  const int pass = tiles ? slot - DPASSES : slot;
  const int need = tiles ? p.tbl->tpasses_needed : p.tbl->dpasses_needed;
  if (pass >= need) return;   // digits zero for every key
  const bool last = pass == need - 1;   // the pass that writes the final order
  const u32 ntiles = p.tbl->total_tiles;
  const int shift = 32 + RADIX_BITS * pass;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  u64 P;
  if (tiles) {
    const u64 Pall = hdr->pairs;
    P = Pall < p.capacity ? Pall : p.capacity;
  } else {
    P = hdr->n_active;
  }
  const u32 tag = hdr->epoch * (u32)MAX_PASSES + (u32)slot;
  {
    const u32 hx = block_excl_scan(tid < RADIX ? p.hist[slot * RADIX + tid] : 0u, S.scratch);
    if (tid < RADIX) S.hist_excl[tid] = hx;
  }
  const u32 lt_mask = (1u << lane) - 1u;
  for (;;) {
    if (tid == 0) S.part = atomicAdd(&hdr->sort_counter[slot], 1u);
    for (int i = tid; i < (SORT_THREADS / 32) * RADIX; i += SORT_THREADS) (&S.warp_cnt[0][0])[i] = 0;
    __syncthreads();
    const u32 part = S.part;
    const u64 base = (u64)part * PART;
    if (base >= P) break;
    u64 key[ITEMS];
    u32 rank[ITEMS];
    const u64 wbase = base + (u64)warp * 32 * ITEMS;
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
      const u64 idx = wbase + (u64)i * 32 + lane;
      const bool valid = idx < P;
      key[i] = valid ? kin[idx] : ~0ull;
    }
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
      const u64 idx = wbase + (u64)i * 32 + lane;
      const bool valid = idx < P;
      const u32 d = (u32)(key[i] >> shift) & (RADIX - 1);
#if GS_SORT_BALLOT_RANK
      // the lanes holding the same digit, one vote per digit bit
      u32 peers = __ballot_sync(0xffffffffu, valid);
#pragma unroll
      for (int b = 0; b < RADIX_BITS; ++b) {
        const u32 v = __ballot_sync(0xffffffffu, (d >> b) & 1u);
        peers &= ((d >> b) & 1u) ? v : ~v;
      }
      const int leader = __ffs(peers) - 1;
      u32 old = 0;
      if (valid && lane == leader) old = atomicAdd(&S.warp_cnt[warp][d], (u32)__popc(peers));
      old = __shfl_sync(0xffffffffu, old, leader & 31);
#else
      const u32 peers = __match_any_sync(0xffffffffu, valid ? d : (RADIX + lane));
      const int leader = __ffs(peers) - 1;
      u32 old = 0;
      if (valid && lane == leader) {
        old = S.warp_cnt[warp][d];
        S.warp_cnt[warp][d] = old + __popc(peers);
      }
      old = __shfl_sync(0xffffffffu, old, leader);
#endif
      rank[i] = old + __popc(peers & lt_mask);
      __syncwarp();
    }
    __syncthreads();
    // digit `tid` (first RADIX threads): exclusive prefix over warps, partition count, look-back
    u32 cnt = 0;
    u64 excl = 0;
    if (tid < RADIX) {
#pragma unroll
      for (int w = 0; w < SORT_THREADS / 32; ++w) {
        const u32 c = S.warp_cnt[w][tid];
        S.warp_cnt[w][tid] = cnt;
        cnt += c;
      }
      u64* st = p.sort_status + (u64)part * RADIX + tid;
      if (part == 0) {
        st_relaxed(st, lb_pack(LB_FLAG_PREFIX, tag, cnt));
      } else {
        st_relaxed(st, lb_pack(LB_FLAG_AGG, tag, cnt));
        excl = lookback_walk(p.sort_status + tid, RADIX, part, tag, hdr, 3 + slot);
        st_relaxed(st, lb_pack(LB_FLAG_PREFIX, tag, excl + cnt));
      }
    }
    const u32 lex = block_excl_scan(tid < RADIX ? cnt : 0u, S.scratch);
    if (tid < RADIX) {
      S.local_excl[tid] = lex;
      S.glob[tid] = S.hist_excl[tid] + (u32)excl - lex;
    }
    __syncthreads();
    // local scatter into shared memory (stable: warp order, round order, lane order)
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
      const u64 idx = wbase + (u64)i * 32 + lane;
      if (idx < P) {
        const u32 d = (u32)(key[i] >> shift) & (RADIX - 1);
        const u32 lp = S.local_excl[d] + S.warp_cnt[warp][d] + rank[i];
        S.keys[lp] = key[i];
      }
    }
    __syncthreads();
    const u32 nvalid = (u32)((P - base) < (u64)PART ? (P - base) : (u64)PART);
    for (u32 j = tid; j < nvalid; j += SORT_THREADS) {
      const u64 k = S.keys[j];
      const u32 d = (u32)(k >> shift) & (RADIX - 1);
      const u32 g = S.glob[d] + j;
      kout[g] = k;
      if (last && tiles) {
        // final positions: this partition's keys of one digit land contiguously and in tile order,
        // so a tile's first (last) key here is one whose shared-memory neighbour has another tile;
        // the tile's range is the least first and the greatest last position over the partitions
        const u32 t = (u32)(k >> 32);
        if (t >= ntiles) {   // cannot happen for keys this frame emitted; guards the table write
          set_status(hdr, GS_ERR_INVALID_ARG);
        } else {
          if (j == 0 || (u32)(S.keys[j - 1] >> 32) != t) atomicMin(&p.ranges[t].x, g);
          if (j + 1 == nvalid || (u32)(S.keys[j + 1] >> 32) != t) atomicMax(&p.ranges[t].y, g + 1);
        }
      } else if (last) {
        // depth ranks: the kept-tile count of the primitive at rank g joins its rank chunk's sum
        // (one add per chunk and warp; a warp's positions are mostly consecutive)
        const u32 chunk = g / SCAN_CHUNK;
        const u32 v = p.touched[(u32)k];
        const u32 peers = __match_any_sync(__activemask(), chunk);
        const u32 sum = __reduce_add_sync(peers, v);
        if (lane == __ffs(peers) - 1 && sum)
          atomicAdd(reinterpret_cast<unsigned long long*>(p.rank_partials + chunk), (unsigned long long)sum);
      }
    }
    __syncthreads();
  }
}

// The compositing kernels' schedule: tiles by descending pair count, bucketed (count / 4, capped),
// so persistent CTAs start the longest lists first and the launch ends on short ones.  One CTA.
constexpr int ORDER_THREADS = 1024, ORDER_BUCKETS = 1024, ORDER_SHIFT = 2;
__global__ void __launch_bounds__(ORDER_THREADS) k_tile_order(WsPtrs p) {
  pdl_begin();
  __shared__ u32 s_off[ORDER_BUCKETS];
  __shared__ u32 s_warp[ORDER_THREADS / 32];
  if (read_status(p.hdr) != 0) return;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const u32 ntiles = p.tbl->total_tiles;
  auto bucket = [](uint2 rg) {   // descending length -> ascending bucket
    const u32 b = (rg.y - rg.x) >> ORDER_SHIFT;
    return (u32)(ORDER_BUCKETS - 1) - (b < (u32)(ORDER_BUCKETS - 1) ? b : (u32)(ORDER_BUCKETS - 1));
  };
  // the ranges the last tile pass left: a tile it never saw is still (~0, 0) and becomes (0, 0);
  // with one tile there is no tile pass and every pair is that tile's
  if (p.tbl->tpasses_needed == 0) {
    if (tid == 0 && ntiles > 0) {
      const u64 Pall = p.hdr->pairs;
      p.ranges[0] = make_uint2(0u, (u32)(Pall < p.capacity ? Pall : p.capacity));
    }
  } else {
    for (u32 t = tid; t < ntiles; t += ORDER_THREADS)
      if (p.ranges[t].x > p.ranges[t].y) p.ranges[t] = make_uint2(0u, 0u);
  }
  s_off[tid] = 0;   // ORDER_THREADS == ORDER_BUCKETS
  __syncthreads();
  for (u32 t = tid; t < ntiles; t += ORDER_THREADS) atomicAdd(&s_off[bucket(p.ranges[t])], 1u);
  __syncthreads();
  // exclusive scan of the bucket counts, one per thread
  const u32 v = s_off[tid];
  u32 incl = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const u32 x = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += x;
  }
  if (lane == 31) s_warp[warp] = incl;
  __syncthreads();
  u32 wbase = 0;
  for (int w = 0; w < warp; ++w) wbase += s_warp[w];
  s_off[tid] = wbase + incl - v;
  __syncthreads();
  for (u32 t = tid; t < ntiles; t += ORDER_THREADS) p.tile_order[atomicAdd(&s_off[bucket(p.ranges[t])], 1u)] = t;
}
static_assert(ORDER_THREADS == ORDER_BUCKETS, "one bucket per thread");

template <int ITEMS>
static int sort_grid(const Launch& L) {
  static int grid = 0;
  if (!grid) {
    const size_t smem = sizeof(SortSmem<ITEMS>);
    if (cudaFuncSetAttribute(k_onesweep<ITEMS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess)
      return -1;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_onesweep<ITEMS>, SORT_THREADS, smem) !=
            cudaSuccess ||
        per_sm < 1)
      per_sm = 1;
    grid = per_sm * L.sm_count;
  }
  return grid;
}

// Passes [first, first + count) of one sort, ping-ponging between b0 and b1 (input in b0); a pass
// with no work leaves its input in place, so the result is in b1 iff the number of working passes is
// odd.  `items` bounds the keys a pass can have.
template <int ITEMS, int GROUP>
static cudaError_t run_passes(const WsPtrs& p, u64* b0, u64* b1, int first, int count, u64 items, const Launch& L) {
  const int sg = sort_grid<ITEMS>(L);
  if (sg < 0) return cudaErrorInvalidValue;
  constexpr int PART = SORT_THREADS * ITEMS;
  const u64 parts = (items + PART - 1) / PART;
  int grid = (u64)sg < parts ? sg : (int)parts;
  if (grid < 1) grid = 1;
  for (int ps = 0; ps < count; ++ps) {
    launch_pdl<GROUP>(k_onesweep<ITEMS>, grid, SORT_THREADS, sizeof(SortSmem<ITEMS>), L.stream, p, b0, b1, first + ps);
    u64* t = b0;
    b0 = b1;
    b1 = t;
  }
  return cudaGetLastError();
}

cudaError_t launch_depth_sort(const FrameTable& tbl, const WsPtrs& p, const Launch& L) {
  return run_passes<DSORT_ITEMS, PDL_DSORT>(p, p.dkeys0, p.dkeys1, 0, DPASSES, tbl.launch_prims, L);
}

cudaError_t launch_bin_sort(const FrameTable& tbl, const WsPtrs& p, const Launch& L) {
  // the tile-digit counts come from the emission; the last tile pass writes the ranges
  if (tbl.tpasses > 0) {
    const cudaError_t e = run_passes<SORT_ITEMS, PDL_TSORT>(p, p.keys0, p.keys1, DPASSES, tbl.tpasses, p.capacity, L);
    if (e != cudaSuccess) return e;
  }
  launch_pdl<PDL_TSORT>(k_tile_order, 1, ORDER_THREADS, 0, L.stream, p);
  return cudaGetLastError();
}

}  // namespace gs
