// Training losses (Sec. 3.4.1): the photometric L1 (or L2) term, and the full objective of Eq. 11,
// (1 - lambda) L1 + lambda D-SSIM, in one fused pass that also writes dL/dimage.
#include "common.cuh"

namespace gs {

constexpr int LOSS_THREADS = 256;

// Neumaier's compensated summation in float32: s + c carries the running sum to about 2^-48.
__device__ __forceinline__ void add_compensated(float& s, float& c, float x) {
  const float t = __fadd_rn(s, x);
  c = __fadd_rn(c, fabsf(s) >= fabsf(x) ? __fadd_rn(__fsub_rn(s, t), x) : __fadd_rn(__fsub_rn(x, t), s));
  s = t;
}

// Sum of one double per thread over a CTA of NTHREADS threads; the result is valid on thread 0.
template <int NTHREADS>
__device__ __forceinline__ double cta_sum(double v, double* s_warp) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) s_warp[threadIdx.x >> 5] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < NTHREADS / 32; ++w) t += s_warp[w];
  return t;
}

// Mean L1 or L2 over `count` values.  Per-element work is float32 (|d| is exact; d^2 adds its
// exact rounding error from an FMA to the compensation term), one float64 per thread at the end:
// the slow float64 pipe sees one addition per thread instead of one per element.
__global__ void __launch_bounds__(LOSS_THREADS) k_loss_partial(const float* __restrict__ img,
                                                              const float* __restrict__ tgt, long long count,
                                                              int kind, float* __restrict__ dL,
                                                              double* __restrict__ partials) {
  pdl_begin();
  __shared__ double s_warp[LOSS_THREADS / 32];
  const double invN = 1.0 / (double)count;
  const float invNf = (float)invN;                   // = (float)(+-1.0 * invN): the same dL bits
  float s = 0.f, c = 0.f;
  // one value: |d| (L1) or d^2 (L2, with the product's rounding error) into the compensated sum
  auto one = [&](float x, float y) -> float {
    const float d = __fsub_rn(x, y);
    if (kind == GS_LOSS_L1) {
      add_compensated(s, c, fabsf(d));
      return d > 0.f ? invNf : (d < 0.f ? -invNf : 0.f);
    }
    const float p = __fmul_rn(d, d);
    add_compensated(s, c, p);
    c = __fadd_rn(c, __fmaf_rn(d, d, -p));
    return (float)(2.0 * (double)d * invN);
  };
  const long long stride = (long long)gridDim.x * LOSS_THREADS;
  const long long i0 = (long long)blockIdx.x * LOSS_THREADS + threadIdx.x;
  const bool vec = ((reinterpret_cast<uintptr_t>(img) | reinterpret_cast<uintptr_t>(tgt) |
                     reinterpret_cast<uintptr_t>(dL)) & 15) == 0;
  long long done = 0;
  if (vec) {   // 16-byte loads and stores over the whole float4s
    const long long n4 = count / 4;
    const float4* a4 = reinterpret_cast<const float4*>(img);
    const float4* b4 = reinterpret_cast<const float4*>(tgt);
    float4* g4 = reinterpret_cast<float4*>(dL);
    for (long long i = i0; i < n4; i += stride) {
      const float4 a = __ldg(a4 + i), b = __ldg(b4 + i);
      float4 g;
      g.x = one(a.x, b.x);
      g.y = one(a.y, b.y);
      g.z = one(a.z, b.z);
      g.w = one(a.w, b.w);
      g4[i] = g;
    }
    done = 4 * n4;
  }
  for (long long i = done + i0; i < count; i += stride) dL[i] = one(img[i], tgt[i]);
  const double t = cta_sum<LOSS_THREADS>((double)s + (double)c, s_warp);
  if (threadIdx.x == 0) partials[blockIdx.x] = t;
}

__global__ void k_loss_final(const double* __restrict__ partials, int n, long long count, double* out) {
  pdl_begin();
  __shared__ double s[256];
  double a = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) a += partials[i];
  s[threadIdx.x] = a;
  __syncthreads();
  for (int st = 128; st; st >>= 1) {
    if ((int)threadIdx.x < st) s[threadIdx.x] += s[threadIdx.x + st];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = s[0] / (double)count;
}

cudaError_t launch_loss(const float* img, const float* tgt, long long count, int kind, double* loss_out, float* dL,
                        double* partials, int nblocks, cudaStream_t s) {
  launch_pdl<PDL_LOSS>(k_loss_partial, nblocks, LOSS_THREADS, 0, s, img, tgt, count, kind, dL, partials);
  launch_pdl<PDL_LOSS>(k_loss_final, 1, 256, 0, s, partials, nblocks, count, loss_out);
  return cudaGetLastError();
}

// ------------------------------------------------------------------------------------------------
// L = (1 - lambda) mean|x - y| + lambda (1 - mean SSIM(x, y)), per channel, SSIM with the 11 x 11
// Gaussian window (sigma 1.5, unit sum), zeros outside the image, C1 = 0.01^2, C2 = 0.03^2.
//
// With s = (a1 a2)/(b1 b2), a1 = 2 mx my + C1, a2 = 2 cov + C2, b1 = mx^2 + my^2 + C1,
// b2 = vx + vy + C2 at pixel p and the moments mx = w*x, vx = w*x^2 - mx^2, cov = w*(xy) - mx my:
//   d(sum_p s)/dx(q) = (w * A)(q) + 2 x(q) (w * B)(q) + y(q) (w * C)(q)
//   B = ds/dvx = -s/b2,  C = ds/dcov = 2 s/a2,  A = ds/dmx - 2 mx B - my C,
//   ds/dmx = s (2 my/a1 - 2 mx/b1),
// the window being symmetric and A = B = C = 0 at pixels outside the image.
//
// One CTA per 32 x 32 output tile of one channel, everything in shared memory:
//   1. the inputs over the tile and a 10-pixel ring;
//   2-3. the five moments, then SSIM and A, B, C, over the tile and a 5-pixel ring;
//   4-5. the window applied to A, B, C over the tile, and the gradient.
// Each separable pass keeps a run of outputs per thread in registers, so one shared-memory load
// feeds up to 11 FMAs.  Row strides are odd and horizontal passes give consecutive lanes
// consecutive rows, so no pass has bank conflicts.  A, B, C overwrite the inputs (step 5 reads x
// and y at the tile's pixels again from global memory), which keeps three CTAs per SM.
// ------------------------------------------------------------------------------------------------
constexpr int SS_T = 32;                      // output tile edge
constexpr int SS_R = 5;                       // window radius
constexpr int SS_K = 2 * SS_R + 1;            // window taps
constexpr int SS_IN = SS_T + 4 * SS_R;        // 52: input rows and columns
constexpr int SS_MID = SS_T + 2 * SS_R;       // 42: rows and columns of the moments and of A, B, C
constexpr int SX = SS_IN + 1;                 // odd row strides (floats)
constexpr int SH = SS_MID + 1;
constexpr int SB = SS_T + 1;
#ifndef GS_SSIM_THREADS
#define GS_SSIM_THREADS 320
#endif
constexpr int SS_THREADS = GS_SSIM_THREADS;
constexpr int SS_IN_FLOATS = 2 * SS_IN * SX;          // x, y; later A, B, C
constexpr int SS_HM_FLOATS = 5 * SS_IN * SH;          // horizontal moments; later the horizontal A, B, C
constexpr size_t SS_SMEM = sizeof(float) * (SS_IN_FLOATS + SS_HM_FLOATS);
static_assert(3 * SS_MID * SH <= SS_IN_FLOATS, "A, B, C reuse the input rows");
static_assert(3 * SS_MID * SB <= SS_HM_FLOATS, "the horizontal pass of A, B, C reuses the moment rows");

struct SsimWindow {
  float w[SS_K];
};

__global__ void __launch_bounds__(SS_THREADS) k_l1_dssim(const float* __restrict__ img, const float* __restrict__ tgt,
                                                        int H, int W, float lambda, double invN, SsimWindow win,
                                                        float* __restrict__ dL, double* __restrict__ partials) {
  pdl_begin();
  extern __shared__ __align__(16) float sm[];
  float* sx = sm;                                  // [IN][SX]
  float* sy = sx + SS_IN * SX;                     // [IN][SX]
  float* am = sm;                                  // [3][MID][SH] A, B, C (after step 2)
  float* hm = sm + SS_IN_FLOATS;                   // [5][IN][SH] horizontal moments
  float* hb = hm;                                  // [3][MID][SB] horizontal pass of A, B, C (after step 3)
  __shared__ double s_warp[SS_THREADS / 32];
  const int tid = threadIdx.x;
  const int x0 = blockIdx.x * SS_T, y0 = blockIdx.y * SS_T;
  const size_t plane = (size_t)H * W;
  const float* X = img + blockIdx.z * plane;
  const float* Y = tgt + blockIdx.z * plane;
  constexpr float C1 = 0.0001f, C2 = 0.0009f;

  // 1. inputs over the tile and a 10-pixel ring, zero outside the image (every load of a thread
  //    issued before the first store, so their latencies overlap)
  {
    constexpr int NL = (SS_IN * SS_IN + SS_THREADS - 1) / SS_THREADS;
    float lx[NL], ly[NL];
#pragma unroll
    for (int k = 0; k < NL; ++k) {
      const int i = tid + k * SS_THREADS;
      const int r = i / SS_IN, q = i - r * SS_IN;
      const int gy = y0 - 2 * SS_R + r, gx = x0 - 2 * SS_R + q;
      const bool in = i < SS_IN * SS_IN && gy >= 0 && gy < H && gx >= 0 && gx < W;
      lx[k] = in ? __ldg(X + (size_t)gy * W + gx) : 0.f;
      ly[k] = in ? __ldg(Y + (size_t)gy * W + gx) : 0.f;
    }
#pragma unroll
    for (int k = 0; k < NL; ++k) {
      const int i = tid + k * SS_THREADS;
      if (i < SS_IN * SS_IN) {
        const int r = i / SS_IN, q = i - r * SS_IN;
        sx[r * SX + q] = lx[k];
        sy[r * SX + q] = ly[k];
      }
    }
  }
  __syncthreads();

  // 2. horizontal window over x, y, x^2, y^2, xy: IN rows x MID columns, 7 outputs per item,
  //    consecutive lanes on consecutive rows
  for (int it = tid; it < SS_IN * 6; it += SS_THREADS) {
    const int c0 = (it / SS_IN) * 7, r = it - (it / SS_IN) * SS_IN;
    const float* px = sx + r * SX + c0;
    const float* py = sy + r * SX + c0;
    float acc[5][7];
#pragma unroll
    for (int m = 0; m < 5; ++m)
#pragma unroll
      for (int o = 0; o < 7; ++o) acc[m][o] = 0.f;
#pragma unroll
    for (int j = 0; j < 7 + 2 * SS_R; ++j) {
      const float u = px[j], v = py[j];
      const float uu = u * u, vv = v * v, uv = u * v;
#pragma unroll
      for (int o = 0; o < 7; ++o) {
        const int k = j - o;
        if (k >= 0 && k < SS_K) {
          const float w = win.w[k];
          acc[0][o] = fmaf(w, u, acc[0][o]);
          acc[1][o] = fmaf(w, v, acc[1][o]);
          acc[2][o] = fmaf(w, uu, acc[2][o]);
          acc[3][o] = fmaf(w, vv, acc[3][o]);
          acc[4][o] = fmaf(w, uv, acc[4][o]);
        }
      }
    }
#pragma unroll
    for (int m = 0; m < 5; ++m)
#pragma unroll
      for (int o = 0; o < 7; ++o) hm[(m * SS_IN + r) * SH + c0 + o] = acc[m][o];
  }
  __syncthreads();

  // 3. vertical window -> moments over MID x MID, then SSIM and A, B, C (6 rows per item,
  //    consecutive lanes on consecutive columns)
  float dssim = 0.f;
  for (int it = tid; it < SS_MID * 7; it += SS_THREADS) {
    const int r0 = (it / SS_MID) * 6, q = it - (it / SS_MID) * SS_MID;
    float acc[5][6];
#pragma unroll
    for (int m = 0; m < 5; ++m)
#pragma unroll
      for (int o = 0; o < 6; ++o) acc[m][o] = 0.f;
#pragma unroll
    for (int j = 0; j < 6 + 2 * SS_R; ++j) {
      float val[5];
#pragma unroll
      for (int m = 0; m < 5; ++m) val[m] = hm[(m * SS_IN + r0 + j) * SH + q];
#pragma unroll
      for (int o = 0; o < 6; ++o) {
        const int k = j - o;
        if (k >= 0 && k < SS_K) {
          const float w = win.w[k];
#pragma unroll
          for (int m = 0; m < 5; ++m) acc[m][o] = fmaf(w, val[m], acc[m][o]);
        }
      }
    }
#pragma unroll
    for (int o = 0; o < 6; ++o) {
      const int r = r0 + o;
      const int gy = y0 - SS_R + r, gx = x0 - SS_R + q;
      float A = 0.f, Bv = 0.f, Cv = 0.f;
      if (gy >= 0 && gy < H && gx >= 0 && gx < W) {
        const float mx = acc[0][o], my = acc[1][o];
        const float vx = acc[2][o] - mx * mx, vy = acc[3][o] - my * my, cv = acc[4][o] - mx * my;
        const float a1 = 2.f * mx * my + C1, a2 = 2.f * cv + C2;
        const float b1 = mx * mx + my * my + C1, b2 = vx + vy + C2;
        const float s = (a1 * a2) / (b1 * b2);
        Bv = -s / b2;
        Cv = 2.f * s / a2;
        A = s * (2.f * my / a1 - 2.f * mx / b1) - 2.f * mx * Bv - my * Cv;
        if (r >= SS_R && r < SS_R + SS_T && q >= SS_R && q < SS_R + SS_T) dssim += 1.f - s;
      }
      am[(0 * SS_MID + r) * SH + q] = A;
      am[(1 * SS_MID + r) * SH + q] = Bv;
      am[(2 * SS_MID + r) * SH + q] = Cv;
    }
  }
  __syncthreads();

  // 4. horizontal window over A, B, C: MID rows x T columns, 8 outputs per item, consecutive
  //    lanes on consecutive rows
  for (int it = tid; it < SS_MID * 4; it += SS_THREADS) {
    const int c0 = (it / SS_MID) * 8, r = it - (it / SS_MID) * SS_MID;
    float acc[3][8];
#pragma unroll
    for (int m = 0; m < 3; ++m)
#pragma unroll
      for (int o = 0; o < 8; ++o) acc[m][o] = 0.f;
#pragma unroll
    for (int j = 0; j < 8 + 2 * SS_R; ++j) {
      float val[3];
#pragma unroll
      for (int m = 0; m < 3; ++m) val[m] = am[(m * SS_MID + r) * SH + c0 + j];
#pragma unroll
      for (int o = 0; o < 8; ++o) {
        const int k = j - o;
        if (k >= 0 && k < SS_K) {
          const float w = win.w[k];
#pragma unroll
          for (int m = 0; m < 3; ++m) acc[m][o] = fmaf(w, val[m], acc[m][o]);
        }
      }
    }
#pragma unroll
    for (int m = 0; m < 3; ++m)
#pragma unroll
      for (int o = 0; o < 8; ++o) hb[(m * SS_MID + r) * SB + c0 + o] = acc[m][o];
  }
  __syncthreads();

  // 5. vertical window over the tile (4 rows per item) and dL/dx
  const float l1w = (float)((1.0 - (double)lambda) * invN), ssw = (float)((double)lambda * invN);
  float l1 = 0.f;
  for (int it = tid; it < SS_T * 8; it += SS_THREADS) {
    const int r0 = (it / SS_T) * 4, q = it - (it / SS_T) * SS_T;
    float acc[3][4];
#pragma unroll
    for (int m = 0; m < 3; ++m)
#pragma unroll
      for (int o = 0; o < 4; ++o) acc[m][o] = 0.f;
#pragma unroll
    for (int j = 0; j < 4 + 2 * SS_R; ++j) {
      float val[3];
#pragma unroll
      for (int m = 0; m < 3; ++m) val[m] = hb[(m * SS_MID + r0 + j) * SB + q];
#pragma unroll
      for (int o = 0; o < 4; ++o) {
        const int k = j - o;
        if (k >= 0 && k < SS_K) {
          const float w = win.w[k];
#pragma unroll
          for (int m = 0; m < 3; ++m) acc[m][o] = fmaf(w, val[m], acc[m][o]);
        }
      }
    }
#pragma unroll
    for (int o = 0; o < 4; ++o) {
      const int gy = y0 + r0 + o, gx = x0 + q;
      if (gy < H && gx < W) {
        const size_t pix = (size_t)gy * W + gx;
        const float x = __ldg(X + pix), y = __ldg(Y + pix);
        const float d = x - y;
        const float dS = acc[0][o] + 2.f * x * acc[1][o] + y * acc[2][o];
        const float g1 = d > 0.f ? l1w : (d < 0.f ? -l1w : 0.f);
        dL[blockIdx.z * plane + pix] = fmaf(-ssw, dS, g1);
        l1 += fabsf(d);
      }
    }
  }
  const double t = cta_sum<SS_THREADS>((1.0 - (double)lambda) * (double)l1 + (double)lambda * (double)dssim, s_warp);
  if (tid == 0) partials[((size_t)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x] = t;
}

size_t l1_dssim_partials(int C, int H, int W) {
  return (size_t)((W + SS_T - 1) / SS_T) * ((H + SS_T - 1) / SS_T) * C;
}

cudaError_t launch_l1_dssim(const float* img, const float* tgt, int C, int H, int W, float lambda, double* loss_out,
                            float* dL, double* partials, cudaStream_t s) {
  const cudaError_t e = cudaFuncSetAttribute(k_l1_dssim, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SS_SMEM);
  if (e != cudaSuccess) return e;
  SsimWindow win;
  double g[SS_K], sum = 0.0;
  for (int k = 0; k < SS_K; ++k) {
    g[k] = exp(-(double)((k - SS_R) * (k - SS_R)) / (2.0 * 1.5 * 1.5));
    sum += g[k];
  }
  for (int k = 0; k < SS_K; ++k) win.w[k] = (float)(g[k] / sum);
  const long long count = (long long)C * H * W;
  const dim3 grid((W + SS_T - 1) / SS_T, (H + SS_T - 1) / SS_T, C);
  launch_pdl<PDL_LOSS>(k_l1_dssim, grid, SS_THREADS, SS_SMEM, s, img, tgt, H, W, lambda, 1.0 / (double)count, win, dL, partials);
  const int n = (int)l1_dssim_partials(C, H, W);
  launch_pdl<PDL_LOSS>(k_loss_final, 1, 256, 0, s, partials, n, count, loss_out);
  return cudaGetLastError();
}

}  // namespace gs
