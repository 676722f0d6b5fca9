// Depth sort of the (tile, primitive) pairs (Sec. 3.1 "sorted by depth", Sec. 3.3.3 tile rasterizer):
// a stable least-significant-digit radix sort of 64-bit keys (tile << 32 | float bits of depth,
// depth > 0 so the bits order like the values) with 32-bit values, restricted to the
// 32 + ceil(log2(tiles)) significant bits.  Each digit pass is one "onesweep" kernel: a CTA ranks
// its partition locally, obtains the global offset of every digit by decoupled look-back over the
// preceding partitions, and scatters through shared memory so global writes are coalesced.
// The digit counts of all passes come from one up-front histogram kernel.  The pair count stays
// on the device; persistent CTAs take partitions in order from an atomic counter.
#include "common.cuh"

namespace gs {

__global__ void __launch_bounds__(256) k_digit_hist(WsPtrs p, int npasses) {
  __shared__ u32 s_h[MAX_PASSES][RADIX];
  if (read_status(p.hdr) != 0) return;
  for (int i = threadIdx.x; i < MAX_PASSES * RADIX; i += blockDim.x) (&s_h[0][0])[i] = 0;
  __syncthreads();
  const u64 P = p.hdr->pairs;
  const u64 n = P < p.capacity ? P : p.capacity;
  const u32 base = p.tbl->depth_base;
  const int dbits = p.tbl->depth_bits;
  const int need = min(npasses, p.tbl->npasses_needed);
  for (u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (u64)gridDim.x * blockDim.x) {
    const u64 v = sort_value(p.keys0[i], base, dbits);
    for (int ps = 0; ps < need; ++ps) atomicAdd(&s_h[ps][(v >> (RADIX_BITS * ps)) & (RADIX - 1)], 1u);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < npasses * RADIX; i += blockDim.x) {
    const u32 c = (&s_h[0][0])[i];
    if (c) atomicAdd(p.hist + i, c);
  }
}

static_assert(SORT_THREADS >= RADIX && SORT_THREADS % 32 == 0, "one digit per thread of the first RADIX threads");

struct SortSmem {
  u32 warp_cnt[SORT_THREADS / 32][RADIX];
  u32 local_excl[RADIX];
  u32 glob[RADIX];
  u32 hist_excl[RADIX];
  u32 scratch[SORT_THREADS / 32];
  u32 part;
  u64 keys[SORT_TILE];
  u32 vals[SORT_TILE];
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

__global__ void __launch_bounds__(SORT_THREADS) k_onesweep(WsPtrs p, const u64* __restrict__ kin,
                                                           const u32* __restrict__ vin, u64* __restrict__ kout,
                                                           u32* __restrict__ vout, int pass, int shift) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  SortSmem& S = *reinterpret_cast<SortSmem*>(smem_raw);
  WsHeader* hdr = p.hdr;
  if (read_status(hdr) != 0) return;
  if (pass >= p.tbl->npasses_needed) return;   // the remaining digits are zero for every key
  const u32 dbase = p.tbl->depth_base;
  const int dbits = p.tbl->depth_bits;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const u64 Pall = hdr->pairs;
  const u64 P = Pall < p.capacity ? Pall : p.capacity;
  const u32 tag = hdr->epoch * (u32)MAX_PASSES + (u32)pass;
  {
    const u32 hx = block_excl_scan(tid < RADIX ? p.hist[pass * RADIX + tid] : 0u, S.scratch);
    if (tid < RADIX) S.hist_excl[tid] = hx;
  }
  const u32 lt_mask = (1u << lane) - 1u;
  for (;;) {
    if (tid == 0) S.part = atomicAdd(&hdr->sort_counter[pass], 1u);
    for (int i = tid; i < (SORT_THREADS / 32) * RADIX; i += SORT_THREADS) (&S.warp_cnt[0][0])[i] = 0;
    __syncthreads();
    const u32 part = S.part;
    const u64 base = (u64)part * SORT_TILE;
    if (base >= P) break;
    u64 key[SORT_ITEMS];
    u32 val[SORT_ITEMS];
    u32 rank[SORT_ITEMS];
    const u64 wbase = base + (u64)warp * 32 * SORT_ITEMS;
#pragma unroll
    for (int i = 0; i < SORT_ITEMS; ++i) {
      const u64 idx = wbase + (u64)i * 32 + lane;
      const bool valid = idx < P;
      key[i] = valid ? kin[idx] : ~0ull;
      val[i] = valid ? vin[idx] : 0u;
    }
#pragma unroll
    for (int i = 0; i < SORT_ITEMS; ++i) {
      const u64 idx = wbase + (u64)i * 32 + lane;
      const bool valid = idx < P;
      const u32 d = (u32)(sort_value(key[i], dbase, dbits) >> shift) & (RADIX - 1);
      const u32 peers = __match_any_sync(0xffffffffu, valid ? d : (RADIX + lane));
      const int leader = __ffs(peers) - 1;
      u32 old = 0;
      if (valid && lane == leader) {
        old = S.warp_cnt[warp][d];
        S.warp_cnt[warp][d] = old + __popc(peers);
      }
      old = __shfl_sync(0xffffffffu, old, leader);
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
        u32 pi = part - 1;
        u32 polls = 0;
        const u64 t0 = global_timer_ns();
        for (;;) {
          const u64 w = ld_relaxed(p.sort_status + (u64)pi * RADIX + tid);
          if (lb_flag(w) != 0 && lb_tag(w) == (tag & 0x3FFFFFu)) {
            excl += lb_value(w);
            if (lb_flag(w) == LB_FLAG_PREFIX) break;
            --pi;  // partition 0 always publishes a prefix
            continue;
          }
          if (++polls > SPIN_LIMIT_POLLS || ((polls & 1023u) == 0 && global_timer_ns() - t0 > SPIN_LIMIT_NS)) {
            hdr->timeout_site = 2 + pass;
            set_status(hdr, GS_ERR_TIMEOUT);
            break;
          }
          __nanosleep(20);
        }
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
    for (int i = 0; i < SORT_ITEMS; ++i) {
      const u64 idx = wbase + (u64)i * 32 + lane;
      if (idx < P) {
        const u32 d = (u32)(sort_value(key[i], dbase, dbits) >> shift) & (RADIX - 1);
        const u32 lp = S.local_excl[d] + S.warp_cnt[warp][d] + rank[i];
        S.keys[lp] = key[i];
        S.vals[lp] = val[i];
      }
    }
    __syncthreads();
    const u32 nvalid = (u32)((P - base) < (u64)SORT_TILE ? (P - base) : (u64)SORT_TILE);
    for (u32 j = tid; j < nvalid; j += SORT_THREADS) {
      const u64 k = S.keys[j];
      const u32 d = (u32)(sort_value(k, dbase, dbits) >> shift) & (RADIX - 1);
      const u32 pos = S.glob[d] + j;
      kout[pos] = k;
      vout[pos] = S.vals[j];
    }
    __syncthreads();
  }
}

__global__ void k_tile_ranges(WsPtrs p) {
  if (read_status(p.hdr) != 0) return;
  const u64* __restrict__ keys = (p.tbl->npasses_needed & 1) ? p.keys1 : p.keys0;
  const u64 Pall = p.hdr->pairs;
  const u64 P = Pall < p.capacity ? Pall : p.capacity;
  const u32 ntiles = p.tbl->total_tiles;
  for (u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x; i < P; i += (u64)gridDim.x * blockDim.x) {
    const u32 t = (u32)(keys[i] >> 32);
    if (t >= ntiles) {   // cannot happen for keys this frame emitted; guards the table write
      set_status(p.hdr, GS_ERR_INVALID_ARG);
      continue;
    }
    if (i == 0 || (u32)(keys[i - 1] >> 32) != t) p.ranges[t].x = (u32)i;
    if (i + 1 == P || (u32)(keys[i + 1] >> 32) != t) p.ranges[t].y = (u32)(i + 1);
  }
}

cudaError_t launch_bin_sort(const FrameTable& tbl, const WsPtrs& p, const Launch& L) {
  static int sort_grid = 0;
  const size_t smem = sizeof(SortSmem);
  if (!sort_grid) {
    cudaError_t e = cudaFuncSetAttribute(k_onesweep, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_onesweep, SORT_THREADS, smem) != cudaSuccess ||
        per_sm < 1)
      per_sm = 1;
    sort_grid = per_sm * L.sm_count;
  }
  const int npasses = tbl.npasses;
  int grid = sort_grid;
  if ((u32)grid > p.n_parts) grid = (int)p.n_parts;
  if (grid < 1) grid = 1;
  k_digit_hist<<<L.sm_count * 4, 256, 0, L.stream>>>(p, npasses);
  const u64* kin = p.keys0;
  const u32* vin = p.vals0;
  u64* kout = p.keys1;
  u32* vout = p.vals1;
  for (int ps = 0; ps < npasses; ++ps) {
    k_onesweep<<<grid, SORT_THREADS, smem, L.stream>>>(p, kin, vin, kout, vout, ps, RADIX_BITS * ps);
    const u64* tk = kout;
    const u32* tv = vout;
    kout = const_cast<u64*>(kin);
    vout = const_cast<u32*>(vin);
    kin = tk;
    vin = tv;
  }
  k_tile_ranges<<<L.sm_count * 8, 256, 0, L.stream>>>(p);
  return cudaGetLastError();
}

}  // namespace gs
