// Frequency-adaptive density control (Sec. 3.4.2; supplement B) on top of the 3DGS rules:
// per-view statistics of the screen-space positional gradient, then clone / split / prune in one
// compaction that resets the frequencies and weights of every new primitive, and the periodic
// reset of opacity and weights.
//
// The compaction is three launches over blocks of DN_THREADS primitives: (1) each block counts its
// kept originals, clones and split primitives; (2) one CTA turns the block counts into block
// offsets of the three output segments and writes the totals; (3) each block recomputes its
// decisions, ranks them inside the block with warp ballots and writes its rows.  Decisions are
// single correctly rounded float32 operations, so they match the written rules bit for bit.
#include "common.cuh"

namespace gs {

constexpr int DN_THREADS = 256;
constexpr int DN_MAX_PRIMS = (1 << 30) - 1;   // 2 n output rows must fit in an int

struct DensifyParams {
  int n, K, nsh, esz;                  // primitives, components, SH coefficients, bytes per SH/Gabor value
  const float* means;
  const float* scales;
  const float* quats;
  const float* opacity;
  const unsigned char* sh;
  const unsigned char* freqs;
  const unsigned char* weights;
  const float* acc;
  const float* den;
  const float* noise;                  // [n][2][3]
  float* o_means;
  float* o_scales;
  float* o_quats;
  float* o_opacity;
  unsigned char* o_sh;
  unsigned char* o_freqs;
  unsigned char* o_weights;
  float grad_threshold, dense_scale, min_opacity, max_scale, split_divisor, child_freq, child_weight;
};

struct Decision {
  bool keep_orig, keep_clone, keep_split;
};

__device__ __forceinline__ Decision densify_decision(const DensifyParams& P, int i) {
  const float s0 = P.scales[3 * i], s1 = P.scales[3 * i + 1], s2 = P.scales[3 * i + 2];
  const float den = P.den[i];
  const float g = den > 0.f ? __fdiv_rn(P.acc[i], den) : 0.f;
  const float smax = fmaxf(fmaxf(s0, s1), s2);
  const bool cand = g >= P.grad_threshold;
  const bool split = cand && smax > P.dense_scale;
  const bool clone = cand && !split;
  const bool low = P.opacity[i] < P.min_opacity;
  const bool big = P.max_scale > 0.f && smax > P.max_scale;
  const float cmax = fmaxf(fmaxf(__fdiv_rn(s0, P.split_divisor), __fdiv_rn(s1, P.split_divisor)),
                           __fdiv_rn(s2, P.split_divisor));
  const bool child_big = P.max_scale > 0.f && cmax > P.max_scale;
  Decision d;
  d.keep_orig = !split && !low && !big;
  d.keep_clone = clone && !low && !big;
  d.keep_split = split && !low && !child_big;
  return d;
}

// Copies `bytes` bytes with the widest unit (16, 8, 4 or 2 bytes) that both addresses and the
// size allow.
__device__ __forceinline__ void copy_row(unsigned char* dst, const unsigned char* src, int bytes) {
  const uintptr_t a = reinterpret_cast<uintptr_t>(dst) | reinterpret_cast<uintptr_t>(src) | (uintptr_t)bytes;
  if ((a & 15) == 0) {
    for (int i = 0; i < bytes / 16; ++i) reinterpret_cast<uint4*>(dst)[i] = reinterpret_cast<const uint4*>(src)[i];
  } else if ((a & 7) == 0) {
    for (int i = 0; i < bytes / 8; ++i) reinterpret_cast<uint2*>(dst)[i] = reinterpret_cast<const uint2*>(src)[i];
  } else if ((a & 3) == 0) {
    for (int i = 0; i < bytes / 4; ++i) reinterpret_cast<u32*>(dst)[i] = reinterpret_cast<const u32*>(src)[i];
  } else {
    for (int i = 0; i < bytes / 2; ++i)
      reinterpret_cast<unsigned short*>(dst)[i] = reinterpret_cast<const unsigned short*>(src)[i];
  }
}

// `count` values of the storage type (float32 or BF16) set to v.
__device__ __forceinline__ void fill_values(unsigned char* dst, int count, int esz, float v) {
  if (esz == 4) {
    for (int i = 0; i < count; ++i) reinterpret_cast<float*>(dst)[i] = v;
  } else {
    const __nv_bfloat16 b = __float2bfloat16_rn(v);
    for (int i = 0; i < count; ++i) reinterpret_cast<__nv_bfloat16*>(dst)[i] = b;
  }
}

// Exclusive ranks of three flags inside the CTA (blockDim.x == DN_THREADS) and the CTA totals.
__device__ __forceinline__ void cta_rank3(const bool f[3], u32 rank[3], u32 total[3]) {
  __shared__ u32 s_w[DN_THREADS / 32][3];
  __shared__ u32 s_base[DN_THREADS / 32][3];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const u32 lt = (1u << lane) - 1u;
  u32 b[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    b[k] = __ballot_sync(0xffffffffu, f[k]);
    if (lane == 0) s_w[warp][k] = __popc(b[k]);
  }
  __syncthreads();
  if (threadIdx.x < 3) {
    u32 run = 0;
    for (int w = 0; w < DN_THREADS / 32; ++w) {
      s_base[w][threadIdx.x] = run;
      run += s_w[w][threadIdx.x];
    }
    s_w[0][threadIdx.x] = run;   // reused as the CTA total once every base is read from s_w
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    rank[k] = s_base[warp][k] + __popc(b[k] & lt);
    total[k] = s_w[0][k];
  }
}

// (1) per-block counts of kept originals, clones and split primitives
__global__ void __launch_bounds__(DN_THREADS) k_densify_count(DensifyParams P, u32* block_counts) {
  pdl_begin();
  const int i = blockIdx.x * DN_THREADS + threadIdx.x;
  bool f[3] = {false, false, false};
  if (i < P.n) {
    const Decision d = densify_decision(P, i);
    f[0] = d.keep_orig;
    f[1] = d.keep_clone;
    f[2] = d.keep_split;
  }
  u32 rank[3], total[3];
  cta_rank3(f, rank, total);
  if (threadIdx.x == 0)
    for (int k = 0; k < 3; ++k) block_counts[3 * blockIdx.x + k] = total[k];
}

// (2) one CTA: exclusive offsets of each block inside the three output segments (in place) and the
//     totals: counts = {all rows, originals, clones, split children}
__global__ void __launch_bounds__(DN_THREADS) k_densify_offsets(u32* block_counts, int nblocks, int* counts) {
  pdl_begin();
  __shared__ u32 s_carry[3];
  if (threadIdx.x < 3) s_carry[threadIdx.x] = 0;
  __syncthreads();
  for (int base = 0; base < nblocks; base += DN_THREADS) {
    const int b = base + threadIdx.x;
    u32 v[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) v[k] = b < nblocks ? block_counts[3 * b + k] : 0u;
    // inclusive scan of v over the CTA, one field at a time (warp shuffles, then warp totals)
    __shared__ u32 s_wsum[DN_THREADS / 32][3];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    u32 inc[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      inc[k] = v[k];
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const u32 t = __shfl_up_sync(0xffffffffu, inc[k], o);
        if (lane >= o) inc[k] += t;
      }
      if (lane == 31) s_wsum[warp][k] = inc[k];
    }
    __syncthreads();
    u32 wbase[3] = {0u, 0u, 0u};
    u32 chunk[3] = {0u, 0u, 0u};
    for (int w = 0; w < DN_THREADS / 32; ++w)
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        if (w < warp) wbase[k] += s_wsum[w][k];
        chunk[k] += s_wsum[w][k];
      }
    if (b < nblocks)
#pragma unroll
      for (int k = 0; k < 3; ++k) block_counts[3 * b + k] = s_carry[k] + wbase[k] + inc[k] - v[k];
    __syncthreads();
    if (threadIdx.x < 3) s_carry[threadIdx.x] += chunk[threadIdx.x];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    counts[1] = (int)s_carry[0];
    counts[2] = (int)s_carry[1];
    counts[3] = (int)(2u * s_carry[2]);
    counts[0] = (int)(s_carry[0] + s_carry[1] + 2u * s_carry[2]);
  }
}

// One output row: attributes of primitive i, with the new-primitive reset and, for a split
// child, the position mu + R(q) (s * z) and scale s / split_divisor.
__device__ __forceinline__ void write_row(const DensifyParams& P, int i, u32 o, bool is_new, int child) {
  const int shb = P.nsh * 3 * P.esz, fb = P.K * 3 * P.esz, wb = P.K * P.esz;
  float m0 = P.means[3 * i], m1 = P.means[3 * i + 1], m2 = P.means[3 * i + 2];
  float s0 = P.scales[3 * i], s1 = P.scales[3 * i + 1], s2 = P.scales[3 * i + 2];
  const float4 q = make_float4(P.quats[4 * i], P.quats[4 * i + 1], P.quats[4 * i + 2], P.quats[4 * i + 3]);
  if (child >= 0) {
    const float inv = 1.f / sqrtf(q.x * q.x + q.y * q.y + q.z * q.z + q.w * q.w);
    const float w = q.x * inv, x = q.y * inv, y = q.z * inv, z = q.w * inv;
    const float* zn = P.noise + 6 * (size_t)i + 3 * child;
    const float v0 = s0 * zn[0], v1 = s1 * zn[1], v2 = s2 * zn[2];
    m0 += (1.f - 2.f * (y * y + z * z)) * v0 + 2.f * (x * y - w * z) * v1 + 2.f * (x * z + w * y) * v2;
    m1 += 2.f * (x * y + w * z) * v0 + (1.f - 2.f * (x * x + z * z)) * v1 + 2.f * (y * z - w * x) * v2;
    m2 += 2.f * (x * z - w * y) * v0 + 2.f * (y * z + w * x) * v1 + (1.f - 2.f * (x * x + y * y)) * v2;
    s0 = __fdiv_rn(s0, P.split_divisor);
    s1 = __fdiv_rn(s1, P.split_divisor);
    s2 = __fdiv_rn(s2, P.split_divisor);
  }
  P.o_means[3 * (size_t)o] = m0;
  P.o_means[3 * (size_t)o + 1] = m1;
  P.o_means[3 * (size_t)o + 2] = m2;
  P.o_scales[3 * (size_t)o] = s0;
  P.o_scales[3 * (size_t)o + 1] = s1;
  P.o_scales[3 * (size_t)o + 2] = s2;
  reinterpret_cast<float4*>(P.o_quats)[o] = q;
  P.o_opacity[o] = P.opacity[i];
  copy_row(P.o_sh + (size_t)o * shb, P.sh + (size_t)i * shb, shb);
  if (is_new) {
    fill_values(P.o_freqs + (size_t)o * fb, P.K * 3, P.esz, P.child_freq);
    fill_values(P.o_weights + (size_t)o * wb, P.K, P.esz, P.child_weight);
  } else if (P.K > 0) {
    copy_row(P.o_freqs + (size_t)o * fb, P.freqs + (size_t)i * fb, fb);
    copy_row(P.o_weights + (size_t)o * wb, P.weights + (size_t)i * wb, wb);
  }
}

// (3) ranks inside the block + block offsets -> rows of the three segments
__global__ void __launch_bounds__(DN_THREADS) k_densify_write(DensifyParams P, const u32* block_offsets,
                                                             const int* counts) {
  pdl_begin();
  const int i = blockIdx.x * DN_THREADS + threadIdx.x;
  Decision d = {false, false, false};
  if (i < P.n) d = densify_decision(P, i);
  const bool f[3] = {d.keep_orig, d.keep_clone, d.keep_split};
  u32 rank[3], total[3];
  cta_rank3(f, rank, total);
  if (i >= P.n) return;
  const u32 n_orig = (u32)counts[1], n_clone = (u32)counts[2];
  if (d.keep_orig) write_row(P, i, block_offsets[3 * blockIdx.x] + rank[0], false, -1);
  if (d.keep_clone) write_row(P, i, n_orig + block_offsets[3 * blockIdx.x + 1] + rank[1], true, -1);
  if (d.keep_split) {
    const u32 o = n_orig + n_clone + 2u * (block_offsets[3 * blockIdx.x + 2] + rank[2]);
    write_row(P, i, o, true, 0);
    write_row(P, i, o + 1u, true, 1);
  }
}

// Statistics of one view: visible primitives (at least one tile this view) add |dL/dmu2D| and one
// visit.  sqrt((gx gx) + (gy gy)) and the sums are single correctly rounded float32 operations.
__global__ void k_densify_accumulate(const u32* __restrict__ touched, int n, const float* __restrict__ grad,
                                     float* __restrict__ acc, float* __restrict__ den) {
  pdl_begin();
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    if (touched[i] == 0) continue;
    const float gx = grad[2 * (size_t)i], gy = grad[2 * (size_t)i + 1];
    acc[i] = __fadd_rn(acc[i], __fsqrt_rn(__fadd_rn(__fmul_rn(gx, gx), __fmul_rn(gy, gy))));
    den[i] = __fadd_rn(den[i], 1.f);
  }
}

cudaError_t launch_densify_accumulate(const u32* touched, int n, const float* grad, float* acc, float* den,
                                      int sm_count, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  int blocks = (n + 255) / 256;
  if (blocks > 8 * sm_count) blocks = 8 * sm_count;
  launch_pdl<PDL_DENSIFY>(k_densify_accumulate, blocks, 256, 0, s, touched, n, grad, acc, den);
  return cudaGetLastError();
}

// The periodic reset: opacity capped at opacity_cap, every weight set to `weight`.
__global__ void k_reset_opacity_weights(float* __restrict__ opacity, unsigned char* __restrict__ weights, int n,
                                        int K, int esz, float opacity_cap, float weight) {
  pdl_begin();
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    opacity[i] = fminf(opacity[i], opacity_cap);
    fill_values(weights + (size_t)i * K * esz, K, esz, weight);
  }
}

}  // namespace gs

using namespace gs;

static bool densify_config_ok(const gs_densify_config* c) {
  return c && isfinite(c->grad_threshold) && isfinite(c->dense_scale) && isfinite(c->min_opacity) &&
         isfinite(c->max_scale) && isfinite(c->split_divisor) && c->split_divisor > 0.f && isfinite(c->child_freq) &&
         isfinite(c->child_weight);
}

static int densify_blocks(int n) { return (n + DN_THREADS - 1) / DN_THREADS; }

extern "C" size_t gabsplat_densify_scratch_bytes(int n) {
  if (n < 0 || n > DN_MAX_PRIMS) return 0;
  return ((size_t)densify_blocks(n) * 3 * sizeof(u32) + 255) / 256 * 256 + 256;
}

extern "C" gs_status gabsplat_densify(const gs_prims* in, const float* grad_accum, const float* denom,
                                      const float* split_noise, const gs_densify_config* cfg,
                                      const gs_prim_arrays* out, long long out_capacity, int* counts, void* scratch,
                                      gs_stream stream) {
  if (!in || !out || !counts || !densify_config_ok(cfg)) return GS_ERR_INVALID_ARG;
  if (in->n < 0 || in->n > DN_MAX_PRIMS || in->K < 0 || in->K > GS_MAX_K || in->sh_degree < 0 ||
      in->sh_degree > GS_MAX_SH_DEGREE || (in->storage != GS_F32 && in->storage != GS_BF16))
    return GS_ERR_INVALID_ARG;
  if (out_capacity < 2LL * in->n) return GS_ERR_INVALID_ARG;   // every primitive yields at most two rows
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (in->n == 0) return cudaMemsetAsync(counts, 0, 4 * sizeof(int), st) == cudaSuccess ? GS_OK : GS_ERR_CUDA;
  if (!in->means || !in->scales || !in->quats || !in->opacity || !in->sh || !grad_accum || !denom || !split_noise ||
      !scratch || !out->means || !out->scales || !out->quats || !out->opacity || !out->sh)
    return GS_ERR_INVALID_ARG;
  if (in->K > 0 && (!in->freqs || !in->weights || !out->freqs || !out->weights)) return GS_ERR_INVALID_ARG;
  if (reinterpret_cast<uintptr_t>(out->quats) & 15) return GS_ERR_INVALID_ARG;
  DensifyParams P;
  P.n = in->n;
  P.K = in->K;
  P.nsh = (in->sh_degree + 1) * (in->sh_degree + 1);
  P.esz = in->storage == GS_BF16 ? 2 : 4;
  P.means = in->means;
  P.scales = in->scales;
  P.quats = in->quats;
  P.opacity = in->opacity;
  P.sh = static_cast<const unsigned char*>(in->sh);
  P.freqs = static_cast<const unsigned char*>(in->freqs);
  P.weights = static_cast<const unsigned char*>(in->weights);
  P.acc = grad_accum;
  P.den = denom;
  P.noise = split_noise;
  P.o_means = out->means;
  P.o_scales = out->scales;
  P.o_quats = out->quats;
  P.o_opacity = out->opacity;
  P.o_sh = static_cast<unsigned char*>(out->sh);
  P.o_freqs = static_cast<unsigned char*>(out->freqs);
  P.o_weights = static_cast<unsigned char*>(out->weights);
  P.grad_threshold = cfg->grad_threshold;
  P.dense_scale = cfg->dense_scale;
  P.min_opacity = cfg->min_opacity;
  P.max_scale = cfg->max_scale;
  P.split_divisor = cfg->split_divisor;
  P.child_freq = cfg->child_freq;
  P.child_weight = cfg->child_weight;
  const int nb = densify_blocks(in->n);
  u32* block_counts = static_cast<u32*>(scratch);
  launch_pdl<PDL_DENSIFY>(k_densify_count, nb, DN_THREADS, 0, st, P, block_counts);
  launch_pdl<PDL_DENSIFY>(k_densify_offsets, 1, DN_THREADS, 0, st, block_counts, nb, counts);
  launch_pdl<PDL_DENSIFY>(k_densify_write, nb, DN_THREADS, 0, st, P, block_counts, counts);
  return cudaGetLastError() == cudaSuccess ? GS_OK : GS_ERR_CUDA;
}

extern "C" gs_status gabsplat_reset_opacity_weights(const gs_prim_arrays* prims, int n, int K, int storage,
                                                    float opacity_cap, float weight, gs_stream stream) {
  if (!prims || n < 0 || n > DN_MAX_PRIMS || K < 0 || K > GS_MAX_K || (storage != GS_F32 && storage != GS_BF16) ||
      !isfinite(opacity_cap) || !isfinite(weight))
    return GS_ERR_INVALID_ARG;
  if (n == 0) return GS_OK;
  if (!prims->opacity || (K > 0 && !prims->weights)) return GS_ERR_INVALID_ARG;
  int blocks = (n + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  launch_pdl<PDL_DENSIFY>(k_reset_opacity_weights, blocks, 256, 0, reinterpret_cast<cudaStream_t>(stream), 
      prims->opacity, static_cast<unsigned char*>(prims->weights), n, K, storage == GS_BF16 ? 2 : 4, opacity_cap,
      weight);
  return cudaGetLastError() == cudaSuccess ? GS_OK : GS_ERR_CUDA;
}
