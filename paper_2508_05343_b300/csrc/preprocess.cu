// Per-primitive stages: frame setup, projection + touched-tile scan + key emission (forward),
// and the chain rule from 2D record gradients to primitive attributes (backward).
//
// Projection follows the paper: envelope Sigma' = J W Sigma W^T J^T with the 2D covariance its
// top-left 2x2 (Sec. 3.1, Eq. 2); frequency f_proj = ((JW)^-1)^T f (Sec. 3.3.1, Eq. 7) and the
// z-integrated 2D frequency f2D = f_proj_xy - (S_02, S_12)/S_22 f_proj_z (Sec. 3.3.2, Eq. 8),
// evaluated here through the equivalent block form f_proj_xy + A^-1 b f_proj_z where A and b are
// the xy block and xz/yz column of the ray-space covariance (-S_xz/S_zz = A^-1 b).  With J's third
// row (0, 0, 1), ((JW)^-1)^T = J^-T W has the closed form used below.
#include "common.cuh"

namespace gs {

// Correctly rounded single operations: the binning quantities (camera depth, projected mean,
// 2D covariance) follow a written float32 procedure with a fixed operation order and no
// fused multiply-add, so tile lists and sort keys are reproducible bit for bit.
#define FM __fmul_rn
#define FA __fadd_rn
#define FS __fsub_rn
#define FDV __fdiv_rn


static_assert(sizeof(FrameTable) + sizeof(WsPtrs) <= 4096, "k_setup parameters must fit the classic 4 KB limit");

__global__ void k_setup(FrameTable tbl, WsPtrs p) {
  pdl_begin();
  const u32* src = reinterpret_cast<const u32*>(&tbl);
  u32* dst = reinterpret_cast<u32*>(const_cast<FrameTable*>(p.tbl));
  for (int i = threadIdx.x; i < (int)(sizeof(FrameTable) / 4); i += blockDim.x) dst[i] = src[i];
  for (int i = threadIdx.x; i < MAX_PASSES * RADIX; i += blockDim.x) p.hist[i] = 0;
  const u32 schunks = (tbl.total_prims + SCAN_CHUNK - 1) / SCAN_CHUNK;   // k_bin adds its active counts
  for (u32 i = threadIdx.x; i < schunks; i += blockDim.x) {   // k_bin and the last depth pass add into these
    p.scan_partials[i] = 0;
    p.rank_partials[i] = 0;
  }
  if (threadIdx.x == 0) {
    WsHeader* h = p.hdr;
    h->status = 0;
    h->epoch = h->epoch + 1;
    h->pairs = 0;
    h->tile_counter_fwd = 0;
    h->tile_counter_bwd = 0;
    h->nonfinite = 0;
    h->timeout_site = 0;
    h->sorted_buf = (u32)(tbl.tpasses_needed & 1);
    h->n_active = 0;
    h->fwd_exits = 0;
    h->bwd_exits = 0;
    h->zero_counter = 0;
    for (int i = 0; i < MAX_PASSES; ++i) h->sort_counter[i] = 0;
  }
}

// Real spherical harmonics up to degree 3 at unit direction (x, y, z); index l*l + l + m.
__device__ __forceinline__ void sh_eval(int deg, float x, float y, float z, float* Y) {
  Y[0] = 0.28209479177387814f;  // 1/(2 sqrt(pi))
  if (deg < 1) return;
  const float c1 = 0.48860251190291992f;  // sqrt(3/(4 pi))
  Y[1] = c1 * y;
  Y[2] = c1 * z;
  Y[3] = c1 * x;
  if (deg < 2) return;
  const float k2a = 1.0925484305920792f;   // sqrt(15/pi)/2
  const float k20 = 0.31539156525252005f;  // sqrt(5/pi)/4
  const float k22 = 0.54627421529603959f;  // sqrt(15/pi)/4
  Y[4] = k2a * x * y;
  Y[5] = k2a * y * z;
  Y[6] = k20 * (3.f * z * z - 1.f);
  Y[7] = k2a * x * z;
  Y[8] = k22 * (x * x - y * y);
  if (deg < 3) return;
  const float k33 = 0.59004358992664352f;   // sqrt(35/(2 pi))/4
  const float k32 = 2.8906114426405538f;    // sqrt(105/pi)/2
  const float k31 = 0.45704579946446572f;   // sqrt(21/(2 pi))/4
  const float k30 = 0.37317633259011540f;   // sqrt(7/pi)/4
  const float k32b = 1.4453057213202769f;   // sqrt(105/pi)/4
  Y[9] = k33 * y * (3.f * x * x - y * y);
  Y[10] = k32 * x * y * z;
  Y[11] = k31 * y * (5.f * z * z - 1.f);
  Y[12] = k30 * z * (5.f * z * z - 3.f);
  Y[13] = k31 * x * (5.f * z * z - 1.f);
  Y[14] = k32b * z * (x * x - y * y);
  Y[15] = k33 * x * (x * x - 3.f * y * y);
}

// Gradient of sum_j Y_j(d) * w_j w.r.t. the direction d (polynomial extension off the sphere;
// its tangential part, the only part used, equals that of the spherical function).
__device__ __forceinline__ void sh_grad(int deg, float x, float y, float z, const float* w, float& gx, float& gy,
                                        float& gz) {
  gx = gy = gz = 0.f;
  if (deg < 1) return;
  const float c1 = 0.48860251190291992f;
  gy += c1 * w[1];
  gz += c1 * w[2];
  gx += c1 * w[3];
  if (deg < 2) return;
  const float k2a = 1.0925484305920792f, k20 = 0.31539156525252005f, k22 = 0.54627421529603959f;
  gx += k2a * y * w[4];
  gy += k2a * x * w[4];
  gy += k2a * z * w[5];
  gz += k2a * y * w[5];
  gz += 6.f * k20 * z * w[6];
  gx += k2a * z * w[7];
  gz += k2a * x * w[7];
  gx += 2.f * k22 * x * w[8];
  gy -= 2.f * k22 * y * w[8];
  if (deg < 3) return;
  const float k33 = 0.59004358992664352f, k32 = 2.8906114426405538f, k31 = 0.45704579946446572f,
              k30 = 0.37317633259011540f, k32b = 1.4453057213202769f;
  gx += 6.f * k33 * x * y * w[9];
  gy += 3.f * k33 * (x * x - y * y) * w[9];
  gx += k32 * y * z * w[10];
  gy += k32 * x * z * w[10];
  gz += k32 * x * y * w[10];
  gy += k31 * (5.f * z * z - 1.f) * w[11];
  gz += 10.f * k31 * y * z * w[11];
  gz += k30 * (15.f * z * z - 3.f) * w[12];
  gx += k31 * (5.f * z * z - 1.f) * w[13];
  gz += 10.f * k31 * x * z * w[13];
  gx += 2.f * k32b * x * z * w[14];
  gy -= 2.f * k32b * y * z * w[14];
  gz += k32b * (x * x - y * y) * w[14];
  gx += 3.f * k33 * (x * x - y * y) * w[15];
  gy -= 6.f * k33 * x * y * w[15];
}

// Binning quantities of one primitive per the float32 specification.
struct BinSpec {
  float tx, ty, tz, mux, muy;
  float Sig[6];         // Sigma: 00 01 02 11 12 22
  float T0[3], T1[3];   // rows of J[0:2] W
  float ux, uy;         // clamped x/z, y/z
  float A00, A01, A11;  // undilated 2D covariance
  double det;           // float64 determinant of the dilated 2D covariance
  bool valid, finite;
  int x0, x1, y0, y1;
};

__device__ __forceinline__ void bin_spec(const ViewDesc& V, float eps2d, float mx, float my, float mz, float s0,
                                         float s1, float s2, float4 q, BinSpec& b) {
  const float* W = V.R;
  b.tx = FA(FA(FA(FM(W[0], mx), FM(W[1], my)), FM(W[2], mz)), V.t[0]);
  b.ty = FA(FA(FA(FM(W[3], mx), FM(W[4], my)), FM(W[5], mz)), V.t[1]);
  b.tz = FA(FA(FA(FM(W[6], mx), FM(W[7], my)), FM(W[8], mz)), V.t[2]);
  const float tx = b.tx, ty = b.ty, tz = b.tz;
  b.mux = FA(FDV(FM(V.fx, tx), tz), V.cx);
  b.muy = FA(FDV(FM(V.fy, ty), tz), V.cy);
  float w = q.x, x = q.y, y = q.z, z = q.w;
  const float nrm = __fsqrt_rn(FA(FA(FA(FM(w, w), FM(x, x)), FM(y, y)), FM(z, z)));
  w = FDV(w, nrm);
  x = FDV(x, nrm);
  y = FDV(y, nrm);
  z = FDV(z, nrm);
  float R[9];
  R[0] = FS(1.f, FM(2.f, FA(FM(y, y), FM(z, z))));
  R[1] = FM(2.f, FS(FM(x, y), FM(w, z)));
  R[2] = FM(2.f, FA(FM(x, z), FM(w, y)));
  R[3] = FM(2.f, FA(FM(x, y), FM(w, z)));
  R[4] = FS(1.f, FM(2.f, FA(FM(x, x), FM(z, z))));
  R[5] = FM(2.f, FS(FM(y, z), FM(w, x)));
  R[6] = FM(2.f, FS(FM(x, z), FM(w, y)));
  R[7] = FM(2.f, FA(FM(y, z), FM(w, x)));
  R[8] = FS(1.f, FM(2.f, FA(FM(x, x), FM(y, y))));
  float M[9];
  const float s[3] = {s0, s1, s2};
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) M[3 * i + j] = FM(R[3 * i + j], s[j]);
  float S[3][3];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = i; j < 3; ++j) {
      S[i][j] = FA(FA(FM(M[3 * i + 0], M[3 * j + 0]), FM(M[3 * i + 1], M[3 * j + 1])), FM(M[3 * i + 2], M[3 * j + 2]));
      S[j][i] = S[i][j];
    }
  b.Sig[0] = S[0][0]; b.Sig[1] = S[0][1]; b.Sig[2] = S[0][2];
  b.Sig[3] = S[1][1]; b.Sig[4] = S[1][2]; b.Sig[5] = S[2][2];
  const float limx = FM(1.3f, FDV(FM(0.5f, (float)V.width), V.fx));
  const float limy = FM(1.3f, FDV(FM(0.5f, (float)V.height), V.fy));
  const float ux = fminf(fmaxf(FDV(tx, tz), -limx), limx);
  const float uy = fminf(fmaxf(FDV(ty, tz), -limy), limy);
  b.ux = ux;
  b.uy = uy;
  const float J00 = FDV(V.fx, tz), J02 = -FDV(FM(V.fx, ux), tz);
  const float J11 = FDV(V.fy, tz), J12 = -FDV(FM(V.fy, uy), tz);
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    b.T0[j] = FA(FM(J00, W[j]), FM(J02, W[6 + j]));
    b.T1[j] = FA(FM(J11, W[3 + j]), FM(J12, W[6 + j]));
  }
  float U0[3], U1[3];
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    U0[j] = FA(FA(FM(b.T0[0], S[0][j]), FM(b.T0[1], S[1][j])), FM(b.T0[2], S[2][j]));
    U1[j] = FA(FA(FM(b.T1[0], S[0][j]), FM(b.T1[1], S[1][j])), FM(b.T1[2], S[2][j]));
  }
  b.A00 = FA(FA(FM(U0[0], b.T0[0]), FM(U0[1], b.T0[1])), FM(U0[2], b.T0[2]));
  b.A01 = FA(FA(FM(U0[0], b.T1[0]), FM(U0[1], b.T1[1])), FM(U0[2], b.T1[2]));
  b.A11 = FA(FA(FM(U1[0], b.T1[0]), FM(U1[1], b.T1[1])), FM(U1[2], b.T1[2]));
  const float ca = FA(b.A00, eps2d), cb = b.A01, cc = FA(b.A11, eps2d);
  // float64 determinant (where near-degenerate footprints cancel); the rest in float32
  const double da = ca, db = cb, dc = cc;
  const double det = __dsub_rn(__dmul_rn(da, dc), __dmul_rn(db, db));
  const float det32 = __double2float_rn(det);
  const float mid = FM(0.5f, FA(ca, cc));
  const float lam = FA(mid, __fsqrt_rn(fmaxf(FS(FM(mid, mid), det32), 0.f)));
  const float rad = ceilf(FM(3.f, __fsqrt_rn(fmaxf(lam, 0.f))));
  b.det = det;
  const float lim = 1073741824.f;   // 2^30
  b.finite = isfinite(b.mux) && isfinite(b.muy) && isfinite(det) && isfinite(rad) && fabsf(b.mux) < lim &&
             fabsf(b.muy) < lim && rad < lim;
  bool valid = (tz > V.znear) && (tz <= V.zfar) && (det > 0.0) && b.finite;
  long long fx0 = 0, fx1 = -1, fy0 = 0, fy1 = -1;
  if (b.finite) {   // floor((mu -+ r) / 16) = floor_div(floor(mu) -+ r, 16), r an integer
    const long long ix = (long long)floorf(b.mux), iy = (long long)floorf(b.muy), ir = (long long)rad;
    fx0 = (ix - ir) >> 4; fx1 = (ix + ir) >> 4;
    fy0 = (iy - ir) >> 4; fy1 = (iy + ir) >> 4;
  }
  valid = valid && fx1 >= 0 && fx0 <= V.tiles_x - 1 && fy1 >= 0 && fy0 <= V.tiles_y - 1;
  b.valid = valid;
  if (valid) {
    b.x0 = (int)(fx0 > 0 ? fx0 : 0);
    b.x1 = (int)(fx1 < V.tiles_x - 1 ? fx1 : V.tiles_x - 1);
    b.y0 = (int)(fy0 > 0 ? fy0 : 0);
    b.y1 = (int)(fy1 < V.tiles_y - 1 ? fy1 : V.tiles_y - 1);
  } else {
    b.x0 = 0; b.x1 = -1; b.y0 = 0; b.y1 = -1;
  }
}

// Tiles a pixel can reach (binning specification): alpha = o G bank <= o G, so a pixel needs the
// squared Mahalanobis distance q <= 2 ln(o / alpha_min).  thr is a float32 upper bound of that
// (frexp and ln m <= (m - 1)/sqrt(m), plus a margin for float32 evaluation).  {q <= thr} is an
// ellipse and the pixel centres of a row of tiles lie in a horizontal strip, so the centres of the
// row it can reach lie in one x-interval, between its leftmost and rightmost points within the
// strip; a tile is kept when its pixel-centre x-range meets that interval (widened slightly).
// Dropped tiles hold only pairs that every pixel skips, so no pixel changes.  Single correctly
// rounded float32 operations in the order the oracle's specification states.
struct Reach {
  float mux, muy;   // projected mean
  float A, B, D;    // conic (A, B, C) and D = A C - B^2
  float thr;        // threshold on q
  float ys;         // y of the ellipse's rightmost point (the leftmost is at -ys)
  float yew;        // y half-extent, widened; < 0: keep every tile of the square's rows
};
constexpr float LN2_UP = 0.693147182464599609375f;   // the float32 just above ln 2
constexpr float PI_SQ = 9.869604401089358f;          // pi^2

__device__ __forceinline__ bool reach_params(const BinSpec& b, float eps2d, float o, float amin, Reach& r) {
  if (!(o >= amin)) return false;
  const float ca = FA(b.A00, eps2d), cb = b.A01, cc = FA(b.A11, eps2d);
  const float det32 = __double2float_rn(b.det);
  const float A = FDV(cc, det32), B = FDV(-cb, det32), C = FDV(ca, det32);
  int e = 0;
  const float m = frexpf(FDV(o, amin), &e);
  const float m2 = FM(m, 2.f);
  const float t = FA(FM((float)(e - 1), LN2_UP), FDV(FS(m2, 1.f), __fsqrt_rn(m2)));
  const float thr = FA(FM(FM(2.f, t), 1.0009765625f), 0.015625f);
  const float D = FS(FM(A, C), FM(B, B));
  const float ye = __fsqrt_rn(FDV(FM(thr, A), D));
  const float xe = __fsqrt_rn(FDV(FM(thr, C), D));
  const float ys = FDV(FM(-B, xe), C);
  const float yew = FA(FM(ye, 1.0009765625f), 0.00390625f);
  const bool ok = D > 0.f && A > 0.f && C > 0.f && isfinite(D) && isfinite(ys) && isfinite(yew);
  r.mux = b.mux;
  r.muy = b.muy;
  r.A = A;
  r.B = B;
  r.D = D;
  r.thr = thr;
  r.ys = ys;
  r.yew = ok ? yew : -1.f;
  return true;
}

// x of the ellipse's boundary at height y: ((-B) y +- sqrt(max(A thr - (D y) y, 0))) / A.
__device__ __forceinline__ float boundary_x(const Reach& r, float y, bool right) {
  const float root = __fsqrt_rn(fmaxf(FS(FM(r.A, r.thr), FM(FM(r.D, y), y)), 0.f));
  const float by = FM(-r.B, y);
  return FDV(right ? FA(by, root) : FS(by, root), r.A);
}

// Kept tiles of row ty of a square whose columns are [x0, x1]: returns their count and sets first.
__device__ __forceinline__ int row_tiles(const Reach& r, int ty, int x0, int x1, int& first) {
  first = x0;
  if (r.yew < 0.f) return x1 - x0 + 1;
  const float by = (float)(TILE * ty);
  const float lo = fmaxf(FS(FA(by, 0.5f), r.muy), -r.yew);
  const float hi = fminf(FS(FA(by, TILE - 0.5f), r.muy), r.yew);
  if (!(lo <= hi)) return 0;
  float xr = boundary_x(r, fminf(fmaxf(r.ys, lo), hi), true);
  float xl = boundary_x(r, fminf(fmaxf(-r.ys, lo), hi), false);
  xr = FA(FA(xr, FM(fabsf(xr), 0.0009765625f)), 0.00390625f);
  xl = FS(FS(xl, FM(fabsf(xl), 0.0009765625f)), 0.00390625f);
  const float a = fmaxf(ceilf(FM(FS(FA(xl, r.mux), 15.5f), 0.0625f)), (float)x0);
  const float b = fminf(floorf(FM(FS(FA(xr, r.mux), 0.5f), 0.0625f)), (float)x1);
  if (!(a <= b)) return 0;
  first = (int)a;
  return (int)(b - a) + 1;
}

// Bin one primitive (the float32 binning specification).  Returns the rows of its 3-sigma square.
__device__ __forceinline__ u32 bin_one(const FrameTable* tbl, u32 gi, const WsPtrs& p, int& x0, int& y0, int& wx,
                                       u32& dbits, u32& tile_base, int& tiles_x, bool& nonfinite, Reach& r) {
  const int v = view_of_prim(tbl, gi);
  const ViewDesc& V = tbl->v[v];
  const u32 k = gi - V.prim_base;
  const float mx = __ldg(V.means + 3 * (size_t)k), my = __ldg(V.means + 3 * (size_t)k + 1),
              mz = __ldg(V.means + 3 * (size_t)k + 2);
  const float s0 = __ldg(V.scales + 3 * (size_t)k), s1 = __ldg(V.scales + 3 * (size_t)k + 1),
              s2 = __ldg(V.scales + 3 * (size_t)k + 2);
  const float4 q = __ldg(reinterpret_cast<const float4*>(V.quats) + k);
  BinSpec b;
  bin_spec(V, tbl->eps2d, mx, my, mz, s0, s1, s2, q, b);
  tile_base = V.tile_base;
  tiles_x = V.tiles_x;
  nonfinite = (b.tz > V.znear) && (b.tz <= V.zfar) && !b.finite;
  if (!b.valid || !reach_params(b, tbl->eps2d, __ldg(V.opacity + k), tbl->alpha_min, r)) {
    x0 = 0; y0 = 0; wx = 1; dbits = 0;
    return 0;
  }
  x0 = b.x0;
  y0 = b.y0;
  wx = b.x1 - b.x0 + 1;
  dbits = __float_as_uint(b.tz);
  return (u32)(b.y1 - b.y0 + 1);   // rows of the 3-sigma square (each culled to an interval later)
}

// a d - b c within a few units in the last place, also under cancellation: Kahan's algorithm
// with a fused multiply-add recovering the rounding error of b c.
__device__ __forceinline__ float det2_kahan(float a, float d, float b, float c) {
  const float w = b * c;
  const float e = fmaf(-b, c, w);   // w - b c, exactly
  const float f = fmaf(a, d, -w);
  return f + e;
}

// The 2D record of one primitive that touches at least one tile (row `row`, its depth rank): conic
// from the float64 determinant, colour, splatted frequencies.  Recomputes the binning quantities
// (bit-identical).
template <int K, int STORAGE>
__device__ __forceinline__ void record_one(const FrameTable* tbl, u32 gi, u32 row, const WsPtrs& p) {
  const int v = view_of_prim(tbl, gi);
  const ViewDesc& V = tbl->v[v];
  const u32 k = gi - V.prim_base;
  const float mx = __ldg(V.means + 3 * (size_t)k), my = __ldg(V.means + 3 * (size_t)k + 1),
              mz = __ldg(V.means + 3 * (size_t)k + 2);
  const float s0 = __ldg(V.scales + 3 * (size_t)k), s1 = __ldg(V.scales + 3 * (size_t)k + 1),
              s2 = __ldg(V.scales + 3 * (size_t)k + 2);
  const float4 q = __ldg(reinterpret_cast<const float4*>(V.quats) + k);
  BinSpec b;
  bin_spec(V, tbl->eps2d, mx, my, mz, s0, s1, s2, q, b);
  // ---- 2D record: conic from the (float64, rounded) determinant, colour, splatted frequencies ----
  const float det32 = __double2float_rn(b.det);
  const float ca = FDV(FA(b.A11, tbl->eps2d), det32), cb = FDV(-b.A01, det32), cc = FDV(FA(b.A00, tbl->eps2d), det32);
  const float op = __ldg(V.opacity + k);

  // colour: SH at the viewing direction, shifted by 0.5 and clamped at 0
  float dxv = mx - V.campos[0], dyv = my - V.campos[1], dzv = mz - V.campos[2];
  const float inv_len = rsqrtf(dxv * dxv + dyv * dyv + dzv * dzv);
  dxv *= inv_len; dyv *= inv_len; dzv *= inv_len;
  float Y[16];
  const int deg = V.sh_degree;
  sh_eval(deg, dxv, dyv, dzv, Y);
  const int nsh = (deg + 1) * (deg + 1);
  float rgb[3] = {0.5f, 0.5f, 0.5f};
  float shc[48];
  load_sh_row<STORAGE>(V.sh, k, nsh, shc);
#pragma unroll
  for (int j = 0; j < 16; ++j) {
    if (j < nsh) {
#pragma unroll
      for (int c = 0; c < 3; ++c) rgb[c] += Y[j] * shc[3 * j + c];
    }
  }
  float rec[rec_floats(K)];
  rec[0] = b.mux; rec[1] = b.muy; rec[2] = ca; rec[3] = cb;
  rec[4] = cc; rec[5] = op; rec[7] = b.tz;
  rec[8] = fmaxf(rgb[0], 0.f); rec[9] = fmaxf(rgb[1], 0.f); rec[10] = fmaxf(rgb[2], 0.f); rec[11] = 0.f;   // slot 11 unused
  float wsum = 0.f;
  if (K > 0) {
    // A^-1 b with A the undilated 2D block and b the xz / yz column of the ray-space covariance
    const float* W = V.R;
    const float Sw0 = b.Sig[0] * W[6] + b.Sig[1] * W[7] + b.Sig[2] * W[8];
    const float Sw1 = b.Sig[1] * W[6] + b.Sig[3] * W[7] + b.Sig[4] * W[8];
    const float Sw2 = b.Sig[2] * W[6] + b.Sig[4] * W[7] + b.Sig[5] * W[8];
    const float bv0 = b.T0[0] * Sw0 + b.T0[1] * Sw1 + b.T0[2] * Sw2;
    const float bv1 = b.T1[0] * Sw0 + b.T1[1] * Sw1 + b.T1[2] * Sw2;
    const float detA = det2_kahan(b.A00, b.A11, b.A01, b.A01);
    float r0 = 0.f, r1 = 0.f;
    if (detA > 0.f) {
      const float idet = 1.f / detA;
      r0 = det2_kahan(b.A11, bv0, b.A01, bv1) * idet;
      r1 = det2_kahan(b.A00, bv1, b.A01, bv0) * idet;
    }
    const float tzfx = b.tz / V.fx, tzfy = b.tz / V.fy;
    // z-attenuation variant: 1/S_22 = c - b^T A^-1 b (the Schur complement of the ray-space
    // covariance [[A, b], [b^T, c]]), the conditional variance along the ray
    const bool zatt = (tbl->flags & GS_FLAG_Z_ATTENUATION) != 0;
    const float sz = zatt ? fmaxf(W[6] * Sw0 + W[7] * Sw1 + W[8] * Sw2 - (bv0 * r0 + bv1 * r1), 0.f) : 0.f;
    float fr[3 * (K > 0 ? K : 1)], wr[K > 0 ? K : 1];
    load_row<STORAGE, 3 * K>(V.freqs, k, fr);
    load_row<STORAGE, K>(V.weights, k, wr);
#pragma unroll
    for (int i = 0; i < K; ++i) {
      const float f0 = fr[3 * i], f1 = fr[3 * i + 1], f2 = fr[3 * i + 2];
      const float g0 = W[0] * f0 + W[1] * f1 + W[2] * f2;
      const float g1 = W[3] * f0 + W[4] * f1 + W[5] * f2;
      const float g2 = W[6] * f0 + W[7] * f1 + W[8] * f2;
      const float fpx = g0 * tzfx, fpy = g1 * tzfy, fpz = g2 + b.ux * g0 + b.uy * g1;
      rec[12 + 2 * i] = fpx + r0 * fpz;
      rec[12 + 2 * i + 1] = fpy + r1 * fpz;
      const float wi = wr[i];
      rec[12 + 2 * K + i] = zatt ? wi * expf(-2.f * PI_SQ * fpz * fpz * sz) : wi;
      wsum += wi;
    }
#pragma unroll
    for (int i = 12 + 3 * K; i < rec_floats(K); ++i) rec[i] = 0.f;
  }
  rec[6] = 1.f - wsum;
  float4* dst = reinterpret_cast<float4*>(p.records + (size_t)row * rec_floats(K));
#pragma unroll
  for (int i = 0; i < rec_floats(K) / 4; ++i) dst[i] = make_float4(rec[4 * i], rec[4 * i + 1], rec[4 * i + 2], rec[4 * i + 3]);
}

// A warp's owners (one per lane) for the flat walk over the rows of their 3-sigma squares, staged in
// shared memory once per group of 32 primitives so each walk step reads its owner's fields with
// vector loads.
struct __align__(16) Owner {
  Reach r;
  u32 excl, xy0, wx, pad;              // xy0 = x0 | y0 << 16 (tile coordinates < 2^16)
  u32 off, rank, tile_base, tiles_x;   // emission: first pair position, depth rank, view tiling
};
__device__ __forceinline__ void stage_owner(Owner& o, u32 excl, int x0, int y0, int wx, const Reach& r, u32 off,
                                            u32 rank, u32 tile_base, int tiles_x) {
  o.r = r;
  o.excl = excl; o.xy0 = (u32)x0 | ((u32)y0 << 16); o.wx = (u32)wx; o.pad = 0;
  o.off = off; o.rank = rank; o.tile_base = tile_base; o.tiles_x = (u32)tiles_x;
}

// Entry j of the warp's flat list of square rows (owner lanes in order, rows top to bottom): the
// owner lane (largest lane whose exclusive start <= j), and the number and first column of the
// row's kept tiles.  Every lane takes part in the shuffles.
struct FlatRow {
  int owner, ty, first, count;
};
__device__ __forceinline__ void flat_row(u32 j, u32 total, u32 my_excl, const Owner* own, FlatRow& f) {
  int lo = 0;
#pragma unroll
  for (int step = 16; step > 0; step >>= 1) {
    const int cand = lo + step;
    if (__shfl_sync(0xffffffffu, my_excl, cand) <= j) lo = cand;
  }
  f.owner = lo;
  f.count = 0;
  f.first = 0;
  f.ty = 0;
  if (j >= total) return;
  const Owner& o = own[lo];
  const int x0 = (int)(o.xy0 & 0xFFFFu);
  f.ty = (int)(o.xy0 >> 16) + (int)(j - o.excl);
  f.count = row_tiles(o.r, f.ty, x0, x0 + (int)o.wx - 1, f.first);
}

// Binning: (1) bin every primitive and count the tiles of its 3-sigma square that a pixel can reach
// (warp-cooperative, no CTA barriers); a primitive with at least one such tile is active and gets a
// depth key; (2) scan of the active flags that lists the active primitives' depth keys in primitive
// order; (3) depth sort of that list (sort.cu), whose positions are the depth ranks; (4) scan of the
// kept-tile counts in rank order, giving each rank its first pair position; (5) emission of the
// kept pairs, warp-cooperative.

// Per-owner counts of kept tiles over the warp's flat list of square rows; returns this lane's count.
__device__ __forceinline__ u32 count_kept(u32 rows_total, u32 my_row_excl, int x0, int y0, int wx, const Reach& rr,
                                          u32* s_cnt, Owner* own, int lane) {
  s_cnt[lane] = 0;
  stage_owner(own[lane], my_row_excl, x0, y0, wx, rr, 0u, 0u, 0u, 1);
  __syncwarp();
  for (u32 base = 0; base < rows_total; base += 32) {
    FlatRow fr;
    flat_row(base + lane, rows_total, my_row_excl, own, fr);
    if (fr.count > 0) atomicAdd(&s_cnt[fr.owner], (u32)fr.count);
  }
  __syncwarp();
  return s_cnt[lane];
}

__device__ __forceinline__ u32 warp_excl_scan(u32 v, int lane, u32& total) {
  u32 incl = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const u32 t = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += t;
  }
  total = __shfl_sync(0xffffffffu, incl, 31);
  return incl - v;
}


// (1) Binning of every primitive (warp-cooperative tile walks): kept-tile counts, the depth key of
// each active primitive at its index, and the active primitives per chunk of SCAN_CHUNK (added
// into scan_partials, cleared by k_setup).
__global__ void __launch_bounds__(BLOCK) k_bin(WsPtrs p) {
  pdl_begin();
  __shared__ u32 s_cnt[BLOCK / 32][32];
  __shared__ Owner s_own[BLOCK / 32][32];
  const FrameTable* tbl = p.tbl;
  WsHeader* hdr = p.hdr;
  if (read_status(hdr) != 0) return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const u32 total = tbl->total_prims;
  // ranges start empty as (~0, 0): the last tile-sort pass lowers .x and raises .y of each tile it
  // finds, and the tile schedule turns the ones still empty into (0, 0)
  for (u32 i = blockIdx.x * BLOCK + threadIdx.x; i < tbl->total_tiles; i += gridDim.x * BLOCK)
    p.ranges[i] = make_uint2(0xFFFFFFFFu, 0u);
  const u32 nwarps = gridDim.x * (BLOCK / 32);
  for (u32 grp = blockIdx.x * (BLOCK / 32) + warp; (u64)grp * 32 < total; grp += nwarps) {
    const u32 gi = grp * 32 + lane;
    int x0 = 0, y0 = 0, wx = 1, tiles_x = 1;
    u32 dbits = 0, tile_base = 0, sq = 0;
    bool nonfinite = false;
    Reach rr;
    rr.mux = rr.muy = rr.A = rr.B = rr.D = rr.thr = rr.ys = rr.yew = 0.f;
    if (gi < total) sq = bin_one(tbl, gi, p, x0, y0, wx, dbits, tile_base, tiles_x, nonfinite, rr);
    if (__any_sync(0xffffffffu, nonfinite) && lane == 0) {
      atomicAdd(&hdr->nonfinite, 1u);
      set_status(hdr, GS_ERR_NONFINITE);
    }
    u32 wsq_total;
    const u32 my_sq_excl = warp_excl_scan(sq, lane, wsq_total);
    const u32 cnt = count_kept(wsq_total, my_sq_excl, x0, y0, wx, rr, s_cnt[warp], s_own[warp], lane);
    __syncwarp();   // the owner table is restaged by the next group
    if (gi < total) {
      p.touched[gi] = cnt;
      // depth in (znear, zfar]: its float bits minus bits(znear) lie in [1, 2^depth_bits)
      if (cnt > 0) p.dkeys1[gi] = ((u64)(dbits - tbl->depth_base) << 32) | gi;
    }
    // active primitives per scan chunk: a group of 32 lies in one chunk (32 divides SCAN_CHUNK)
    const u32 nact = __popc(__ballot_sync(0xffffffffu, gi < total && cnt > 0));
    if (lane == 0 && nact) atomicAdd(reinterpret_cast<unsigned long long*>(p.scan_partials + grp * 32 / SCAN_CHUNK),
                                     (unsigned long long)nact);
  }
}


// The two scans below run as reduce-then-scan: one launch writes each 4096-element chunk's sum, the
// next adds up its chunk's predecessors directly and scans the chunk.  With about as many chunks as
// resident CTAs, a single-pass look-back would walk back through almost every chunk before it.

// Sum over the CTA of one value per thread (every thread gets the sum).
__device__ __forceinline__ u64 block_sum(u64 v, u64* s_red /*BLOCK / 32*/) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if (lane == 0) s_red[warp] = v;
  __syncthreads();
  u64 t = 0;
#pragma unroll
  for (int w = 0; w < BLOCK / 32; ++w) t += s_red[w];
  __syncthreads();
  return t;
}

// Exclusive scan over the CTA of one value per thread (thread t owns SCAN_ITEMS consecutive items),
// offset by the sum of the partials of the chunks before `chunk`.  Returns the thread's exclusive
// prefix; the chunk's total is left in s_tot.
__device__ __forceinline__ u64 chunk_scan(u32 sum, const u64* partial, u32 chunk, u32* s_warp, u64* s_red,
                                          u64& s_tot) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  u64 before = 0;
  for (u32 c = tid; c < chunk; c += BLOCK) before += partial[c];
  before = block_sum(before, s_red);
  u32 wtot;
  const u32 wex = warp_excl_scan(sum, lane, wtot);
  if (lane == 31) s_warp[warp] = wex + sum;
  __syncthreads();
  if (warp == 0) {
    const u32 wv = lane < BLOCK / 32 ? s_warp[lane] : 0u;
    u32 wt;
    const u32 wx = warp_excl_scan(wv, lane, wt);
    if (lane < BLOCK / 32) s_warp[lane] = wx;
    if (lane == 0) s_tot = wt;
  }
  __syncthreads();
  return before + s_warp[warp] + wex;
}

// (2b) Active list: the primitives with at least one kept tile and their depth keys, in primitive
// order, and the digit counts of the depth sort.  Publishes n_active.
__global__ void __launch_bounds__(BLOCK) k_scan_active(WsPtrs p) {
  pdl_begin();
  __shared__ u32 s_warp[BLOCK / 32];
  __shared__ u64 s_red[BLOCK / 32];
  __shared__ u64 s_tot;
  __shared__ u32 s_h[DPASSES][RADIX];
  const FrameTable* tbl = p.tbl;
  WsHeader* hdr = p.hdr;
  if (read_status(hdr) != 0) return;
  const int tid = threadIdx.x;
  const u32 total = tbl->total_prims;
  const u32 chunk = blockIdx.x;
  const u64 base = (u64)chunk * SCAN_CHUNK;
  if (base >= total) return;
  const int need = tbl->dpasses_needed;
  for (int i = tid; i < DPASSES * RADIX; i += BLOCK) (&s_h[0][0])[i] = 0;
  const u64 my0 = base + (u64)tid * SCAN_ITEMS;
  u32 flags = 0;
#pragma unroll
  for (int i = 0; i < SCAN_ITEMS; ++i)
    if (my0 + i < total && p.touched[my0 + i] > 0) flags |= 1u << i;
  u64 key[SCAN_ITEMS];   // loaded before any store, so the loads overlap
#pragma unroll
  for (int i = 0; i < SCAN_ITEMS; ++i) key[i] = (flags >> i) & 1u ? p.dkeys1[my0 + i] : 0ull;
  u64 run = chunk_scan((u32)__popc(flags), p.scan_partials, chunk, s_warp, s_red, s_tot);
  if (tid == 0 && base + SCAN_CHUNK >= total) hdr->n_active = (u32)(run + s_tot);   // thread 0's prefix is the chunk's
#pragma unroll
  for (int i = 0; i < SCAN_ITEMS; ++i) {
    if ((flags >> i) & 1u) {
      p.active[run] = (u32)(my0 + i);
      p.dkeys0[run++] = key[i];
      for (int ps = 0; ps < need; ++ps)
        atomicAdd(&s_h[ps][(u32)(key[i] >> (32 + RADIX_BITS * ps)) & (RADIX - 1)], 1u);
    }
  }
  __syncthreads();
  for (int i = tid; i < need * RADIX; i += BLOCK) {
    const u32 c = (&s_h[0][0])[i];
    if (c) atomicAdd(p.hist + i, c);
  }
}

// (4b) Rank order: order[r] = the primitive of depth rank r, rank_of[order[r]] = r, offsets[r] = its
// first pair position (exclusive scan of the kept-tile counts in rank order).  Publishes the pair
// count and checks the pair capacity.
__global__ void __launch_bounds__(BLOCK) k_scan_ranked(WsPtrs p) {
  pdl_begin();
  __shared__ u32 s_warp[BLOCK / 32];
  __shared__ u64 s_red[BLOCK / 32];
  __shared__ u64 s_tot;
  const FrameTable* tbl = p.tbl;
  WsHeader* hdr = p.hdr;
  if (read_status(hdr) != 0) return;
  const int tid = threadIdx.x;
  const u32 total = hdr->n_active;
  const u32 chunk = blockIdx.x;
  const u64 base = (u64)chunk * SCAN_CHUNK;
  if (base >= total) return;
  const u64* __restrict__ sorted = (tbl->dpasses_needed & 1) ? p.dkeys1 : p.dkeys0;
  const u64 my0 = base + (u64)tid * SCAN_ITEMS;
  // all loads first (keys, then the counts they index), then the stores: the loads overlap
  u32 gi[SCAN_ITEMS], v[SCAN_ITEMS], sum = 0;
#pragma unroll
  for (int i = 0; i < SCAN_ITEMS; ++i) gi[i] = my0 + i < total ? (u32)sorted[my0 + i] : 0xFFFFFFFFu;
#pragma unroll
  for (int i = 0; i < SCAN_ITEMS; ++i) v[i] = gi[i] != 0xFFFFFFFFu ? p.touched[gi[i]] : 0u;
#pragma unroll
  for (int i = 0; i < SCAN_ITEMS; ++i) {
    sum += v[i];
    if (gi[i] != 0xFFFFFFFFu) {
      p.order[my0 + i] = gi[i];
      p.rank_of[gi[i]] = (u32)(my0 + i);
    }
  }
  u64 run = chunk_scan(sum, p.rank_partials, chunk, s_warp, s_red, s_tot);
  if (tid == 0 && base + SCAN_CHUNK >= total) {   // last chunk: publish the pair count
    const u64 P = run + s_tot;                      // thread 0's prefix is the chunk's
    hdr->pairs = P;
    if (P > p.capacity) set_status(hdr, GS_ERR_CAPACITY);
  }
#pragma unroll
  for (int i = 0; i < SCAN_ITEMS; ++i) {
    if (my0 + i < total) p.offsets[my0 + i] = (u32)run;
    run += v[i];
  }
}

// (5) Emission over the active list (index order, so a warp's 32 primitives mix near and far ones
// and its walk stays balanced): each lane re-bins its own primitive (bit-identical), the warp walks
// the flat list of the owners' square rows 32 at a time, gets each row's kept tiles as an interval,
// and then writes tile << 32 | rank for the kept tiles of those 32 rows, 32 at a time, at
// offsets[rank] + the tile's index among the owner's kept tiles (row-major).
__global__ void __launch_bounds__(BLOCK) k_emit(WsPtrs p) {
  pdl_begin();
  __shared__ u32 s_run[BLOCK / 32][32];
  __shared__ Owner s_own[BLOCK / 32][32];
  __shared__ u32 s_th[MAX_PASSES - DPASSES][RADIX];   // tile-sort digit counts of this CTA's pairs
  const FrameTable* tbl = p.tbl;
  WsHeader* hdr = p.hdr;
  if (read_status(hdr) != 0) return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const u32 nact = hdr->n_active;
  const int tneed = tbl->tpasses_needed;
  for (int i = threadIdx.x; i < (MAX_PASSES - DPASSES) * RADIX; i += BLOCK) (&s_th[0][0])[i] = 0;
  __syncthreads();
  const u32 nwarps = gridDim.x * (BLOCK / 32);
  for (u32 grp = blockIdx.x * (BLOCK / 32) + warp; (u64)grp * 32 < nact; grp += nwarps) {
    const u32 ia = grp * 32 + lane;
    const u32 gi = ia < nact ? p.active[ia] : 0u;
    const u32 rank = ia < nact ? p.rank_of[gi] : 0u;
    int x0 = 0, y0 = 0, wx = 1, tiles_x = 1;
    u32 dbits = 0, tile_base = 0, rows = 0;
    bool nonfinite = false;
    Reach rr;
    rr.mux = rr.muy = rr.A = rr.B = rr.D = rr.thr = rr.ys = rr.yew = 0.f;
    if (ia < nact) rows = bin_one(tbl, gi, p, x0, y0, wx, dbits, tile_base, tiles_x, nonfinite, rr);
    const u32 off = ia < nact ? p.offsets[rank] : 0u;
    u32 rows_total;
    const u32 my_row_excl = warp_excl_scan(rows, lane, rows_total);
    s_run[warp][lane] = 0;
    stage_owner(s_own[warp][lane], my_row_excl, x0, y0, wx, rr, off, rank, tile_base, tiles_x);
    __syncwarp();
    for (u32 base = 0; base < rows_total; base += 32) {
      FlatRow fr;
      flat_row(base + lane, rows_total, my_row_excl, s_own[warp], fr);
      // the tile sort's digit counts above the lowest digit: a row's kept tiles are consecutive, so
      // a higher digit changes at most a few times along them (one add per run)
      if (fr.count > 0) {
        const Owner& o = s_own[warp][fr.owner];
        const u32 t0 = o.tile_base + (u32)fr.ty * o.tiles_x + (u32)fr.first, t1 = t0 + (u32)fr.count;
        for (int ps = 1; ps < tneed; ++ps) {
          const int sh = RADIX_BITS * ps;
          for (u32 a = t0; a < t1;) {
            const u32 b = min(t1, ((a >> sh) + 1u) << sh);
            atomicAdd(&s_th[ps][(a >> sh) & (RADIX - 1)], b - a);
            a = b;
          }
        }
      }
      // this row's first pair position: the owner's kept tiles in earlier rows (earlier steps, and
      // earlier lanes of this step)
      u32 tot;
      const u32 ex = warp_excl_scan((u32)fr.count, lane, tot);
      const u32 peers = __match_any_sync(0xffffffffu, base + lane < rows_total ? fr.owner : 32 + lane);
      const int lead = __ffs(peers) - 1;
      const u32 pos0 = s_own[warp][fr.owner].off + s_run[warp][fr.owner] + ex - __shfl_sync(0xffffffffu, ex, lead);
      __syncwarp();
      if (fr.count > 0) atomicAdd(&s_run[warp][fr.owner], (u32)fr.count);
      // the kept tiles of these 32 rows, one per lane
      for (u32 e0 = 0; e0 < tot; e0 += 32) {
        const u32 e = e0 + lane;
        int src = 0;   // the row lane holding entry e: the largest lane whose exclusive start <= e
#pragma unroll
        for (int step = 16; step > 0; step >>= 1) {
          const int cand = src + step;
          if (__shfl_sync(0xffffffffu, ex, cand) <= e) src = cand;
        }
        const u32 k = e - __shfl_sync(0xffffffffu, ex, src);
        const int ty = __shfl_sync(0xffffffffu, fr.ty, src);
        const int first = __shfl_sync(0xffffffffu, fr.first, src);
        const int owner = __shfl_sync(0xffffffffu, fr.owner, src);
        const u32 pos = __shfl_sync(0xffffffffu, pos0, src) + k;
        u32 tile = 0;
        if (e < tot) {
          const Owner& o = s_own[warp][owner];
          tile = o.tile_base + (u32)ty * o.tiles_x + (u32)(first + (int)k);
          if (pos < p.capacity) p.keys0[pos] = ((u64)tile << 32) | o.rank;
        }
        // the lowest digit, one add per pair (the warp's pairs are mostly consecutive tiles)
        if (e < tot && tneed > 0) atomicAdd(&s_th[0][tile & (RADIX - 1)], 1u);
      }
      __syncwarp();
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < tneed * RADIX; i += BLOCK) {
    const u32 c = (&s_th[0][0])[i];
    if (c) atomicAdd(p.hist + DPASSES * RADIX + i, c);
  }
}

// Resident CTAs per SM that the record and gradient-chain kernels are compiled for.  Both are
// latency-bound over scattered attribute rows, so occupancy matters more than a few spilled registers.
#ifndef GS_RECORDS_MIN_CTAS
#define GS_RECORDS_MIN_CTAS 2
#endif
#ifndef GS_PBWD_MIN_CTAS
#define GS_PBWD_MIN_CTAS 2
#endif

// 2D records of the active primitives (full warps over the active list), each at its depth rank.
template <int K, int STORAGE>
__global__ void __launch_bounds__(BLOCK, GS_RECORDS_MIN_CTAS) k_records(WsPtrs p) {
  pdl_begin();
  if (read_status(p.hdr) != 0) return;
  const u32 n = p.hdr->n_active;
  for (u32 i = blockIdx.x * BLOCK + threadIdx.x; i < n; i += gridDim.x * BLOCK) {
    const u32 gi = p.active[i];
    record_one<K, STORAGE>(p.tbl, gi, p.rank_of[gi], p);
  }
}

// Zero every attribute gradient (culled primitives keep zeros; active ones are overwritten).
__device__ __forceinline__ void zero_fill(float* a, size_t count, size_t tid, size_t nthreads) {
  if (!a) return;
  size_t head = (16 - (reinterpret_cast<uintptr_t>(a) & 15)) / 4 % 4;   // floats before 16-byte alignment
  if (head > count) head = count;
  for (size_t i = tid; i < head; i += nthreads) a[i] = 0.f;
  float4* v = reinterpret_cast<float4*>(a + head);
  const size_t n4 = (count - head) / 4;
  for (size_t i = tid; i < n4; i += nthreads) v[i] = make_float4(0.f, 0.f, 0.f, 0.f);
  for (size_t i = head + 4 * n4 + tid; i < count; i += nthreads) a[i] = 0.f;
}

__global__ void k_zero_grads(gs_prim_grads G, int n, int K, int nsh) {
  pdl_begin();
  const size_t tid = (size_t)blockIdx.x * blockDim.x + threadIdx.x, nt = (size_t)gridDim.x * blockDim.x;
  zero_fill(G.means, 3 * (size_t)n, tid, nt);
  zero_fill(G.scales, 3 * (size_t)n, tid, nt);
  zero_fill(G.quats, 4 * (size_t)n, tid, nt);
  zero_fill(G.opacity, (size_t)n, tid, nt);
  zero_fill(G.sh, (size_t)n * nsh * 3, tid, nt);
  zero_fill(G.freqs, (size_t)n * K * 3, tid, nt);
  zero_fill(G.weights, (size_t)n * K, tid, nt);
  zero_fill(G.means2d, 2 * (size_t)n, tid, nt);
}

ZeroJob make_zero_job(const gs_prim_grads& g, int n, int K, int nsh, u32 ntiles) {
  ZeroJob z{};
  float* const a[ZERO_ARRAYS] = {g.means, g.scales, g.quats, g.opacity, g.sh, g.freqs, g.weights, g.means2d};
  const u64 per[ZERO_ARRAYS] = {3, 3, 4, 1, 3 * (u64)nsh, 3 * (u64)K, (u64)K, 2};
  u64 chunks = 0;
  for (int i = 0; i < ZERO_ARRAYS; ++i) {
    z.a[i] = a[i];
    z.n[i] = a[i] && n > 0 ? per[i] * (u64)n : 0;
    z.base[i] = (u32)chunks;
    chunks += (z.n[i] + ZERO_CHUNK - 1) / ZERO_CHUNK;
  }
  z.base[ZERO_ARRAYS] = (u32)chunks;
  const u64 spread = (u64)ntiles * GS_ZERO_SPREAD_PCT / 100 > 0 ? (u64)ntiles * GS_ZERO_SPREAD_PCT / 100 : 1;
  z.quota = chunks ? (u32)((chunks + spread - 1) / spread) : 0;
  return z;
}

// ------------------------------------------------------------------------------------------
// Backward: 2D record gradients -> primitive attribute gradients (exact chain rule of the
// forward above; clamps pass zero gradient).
// ------------------------------------------------------------------------------------------

template <int K, int STORAGE>
__global__ void __launch_bounds__(BLOCK, GS_PBWD_MIN_CTAS) k_preprocess_bwd(WsPtrs p, gs_prim_grads G) {
  pdl_begin();
  const FrameTable* tbl = p.tbl;
  if (read_status(p.hdr) != 0) return;
  const ViewDesc& V = tbl->v[0];
  const int deg = V.sh_degree;
  const int nsh = (deg + 1) * (deg + 1);
  const u32 n_act = p.hdr->n_active;
  for (u32 ia = blockIdx.x * BLOCK + threadIdx.x; ia < n_act; ia += gridDim.x * BLOCK) {
    const u32 gi = p.active[ia];
    const u32 row = p.rank_of[gi];   // grad2d rows are depth ranks
    const int k = (int)(gi - V.prim_base);
    float g2[g2d_floats(K)];
    {
      const float4* src = reinterpret_cast<const float4*>(p.grad2d + (size_t)row * g2d_floats(K));
#pragma unroll
      for (int i = 0; i < g2d_floats(K) / 4; ++i) {
        const float4 t = src[i];
        g2[4 * i] = t.x; g2[4 * i + 1] = t.y; g2[4 * i + 2] = t.z; g2[4 * i + 3] = t.w;
      }
    }
    float gmean[3] = {0.f, 0.f, 0.f}, gscale[3] = {0.f, 0.f, 0.f}, gquat[4] = {0.f, 0.f, 0.f, 0.f};
    if (G.opacity) G.opacity[k] = g2[5];
    if (G.means2d) store_row<2>(G.means2d, k, g2);
    const float mx = __ldg(V.means + 3 * (size_t)k), my = __ldg(V.means + 3 * (size_t)k + 1),
                mz = __ldg(V.means + 3 * (size_t)k + 2);
    const float s[3] = {__ldg(V.scales + 3 * (size_t)k), __ldg(V.scales + 3 * (size_t)k + 1),
                        __ldg(V.scales + 3 * (size_t)k + 2)};
    const float4 q4 = __ldg(reinterpret_cast<const float4*>(V.quats) + k);
    const float* W = V.R;
    const float eps = tbl->eps2d;
    // ---- recompute forward intermediates ----
    const float tx = W[0] * mx + W[1] * my + W[2] * mz + V.t[0];
    const float ty = W[3] * mx + W[4] * my + W[5] * mz + V.t[1];
    const float tz = W[6] * mx + W[7] * my + W[8] * mz + V.t[2];
    const float qn = sqrtf(q4.x * q4.x + q4.y * q4.y + q4.z * q4.z + q4.w * q4.w);
    const float iqn = 1.f / qn;
    const float qw = q4.x * iqn, qx = q4.y * iqn, qy = q4.z * iqn, qz = q4.w * iqn;
    float R[9];
    R[0] = 1.f - 2.f * (qy * qy + qz * qz); R[1] = 2.f * (qx * qy - qw * qz); R[2] = 2.f * (qx * qz + qw * qy);
    R[3] = 2.f * (qx * qy + qw * qz); R[4] = 1.f - 2.f * (qx * qx + qz * qz); R[5] = 2.f * (qy * qz - qw * qx);
    R[6] = 2.f * (qx * qz - qw * qy); R[7] = 2.f * (qy * qz + qw * qx); R[8] = 1.f - 2.f * (qx * qx + qy * qy);
    float M[9];
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) M[3 * i + j] = R[3 * i + j] * s[j];
    float Sg[9];
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) Sg[3 * i + j] = M[3 * i] * M[3 * j] + M[3 * i + 1] * M[3 * j + 1] + M[3 * i + 2] * M[3 * j + 2];
    const float ifx = 1.f / V.fx, ify = 1.f / V.fy;
    const float limx = 1.3f * (0.5f * (float)V.width / V.fx), limy = 1.3f * (0.5f * (float)V.height / V.fy);
    const float rux = tx / tz, ruy = ty / tz;
    const bool clx = (rux < -limx) || (rux > limx), cly = (ruy < -limy) || (ruy > limy);
    const float ux = fminf(fmaxf(rux, -limx), limx), uy = fminf(fmaxf(ruy, -limy), limy);
    const float J00 = V.fx / tz, J02 = -V.fx * ux / tz, J11 = V.fy / tz, J12 = -V.fy * uy / tz;
    float T0[3], T1[3], w3[3];
    for (int j = 0; j < 3; ++j) {
      T0[j] = J00 * W[j] + J02 * W[6 + j];
      T1[j] = J11 * W[3 + j] + J12 * W[6 + j];
      w3[j] = W[6 + j];
    }
    float U0[3], U1[3], Sw[3];   // U_a = Sigma T_a (Sigma symmetric), Sw = Sigma w3
    for (int i = 0; i < 3; ++i) {
      U0[i] = Sg[3 * i] * T0[0] + Sg[3 * i + 1] * T0[1] + Sg[3 * i + 2] * T0[2];
      U1[i] = Sg[3 * i] * T1[0] + Sg[3 * i + 1] * T1[1] + Sg[3 * i + 2] * T1[2];
      Sw[i] = Sg[3 * i] * w3[0] + Sg[3 * i + 1] * w3[1] + Sg[3 * i + 2] * w3[2];
    }
    const float A00 = U0[0] * T0[0] + U0[1] * T0[1] + U0[2] * T0[2];
    const float A01 = U0[0] * T1[0] + U0[1] * T1[1] + U0[2] * T1[2];
    const float A11 = U1[0] * T1[0] + U1[1] * T1[1] + U1[2] * T1[2];
    const float bv0 = T0[0] * Sw[0] + T0[1] * Sw[1] + T0[2] * Sw[2];
    const float bv1 = T1[0] * Sw[0] + T1[1] * Sw[1] + T1[2] * Sw[2];
    // dilated 2D covariance inverse (conic); the determinants here feed gradients only, so float32
    // with Kahan's compensated 2x2 determinant stands in for the forward's float64 one
    const float ea = A00 + eps, eb = A01, ec = A11 + eps;
    const float idet = 1.f / det2_kahan(ea, ec, eb, eb);
    const float Qa = ec * idet, Qb = -eb * idet, Qc = ea * idet;
    // ---- conic -> 2D covariance: dSigma2D = -Q G Q with G = [[ga, gb/2], [gb/2, gc]] ----
    const float ga = g2[2], gbh = 0.5f * g2[3], gc = g2[4];
    const float QG00 = Qa * ga + Qb * gbh, QG01 = Qa * gbh + Qb * gc;
    const float QG10 = Qb * ga + Qc * gbh, QG11 = Qb * gbh + Qc * gc;
    float gA00 = -(QG00 * Qa + QG01 * Qb);
    float gA11 = -(QG10 * Qb + QG11 * Qc);
    float gA01 = -2.f * (QG00 * Qb + QG01 * Qc);   // the off-diagonal entry appears twice
    float gtx = 0.f, gty = 0.f, gtz = 0.f, gux = 0.f, guy = 0.f;
    float gb0 = 0.f, gb1 = 0.f, gcz = 0.f;   // gcz: dL/d(w3^T Sigma w3), the variant only
    if (K > 0) {
      const float detA = det2_kahan(A00, A11, A01, A01);
      float iA00 = 0.f, iA01 = 0.f, iA11 = 0.f, r0 = 0.f, r1 = 0.f;
      if (detA > 0.f) {
        const float id = 1.f / detA;
        iA00 = A11 * id; iA01 = -A01 * id; iA11 = A00 * id;
        r0 = det2_kahan(A11, bv0, A01, bv1) * id;
        r1 = det2_kahan(A00, bv1, A01, bv0) * id;
      }
      float gr0 = 0.f, gr1 = 0.f;
      const float tzfx = tz * ifx, tzfy = tz * ify;
      // the bank's weight terms: G_i = dL/d(cosine weight i), G0 = dL/d(1 - sum w); in the
      // z-attenuation variant the cosine weight is w_i C2_i, C2_i = exp(-2 pi^2 fpz_i^2 sz) with
      // sz = c - b^T A^-1 b (clamped at 0), else C2_i = 1
      const float G0 = g2[9 + 3 * K];
      const bool zatt = (tbl->flags & GS_FLAG_Z_ATTENUATION) != 0;
      const float sz_raw = zatt ? (w3[0] * Sw[0] + w3[1] * Sw[1] + w3[2] * Sw[2]) - (bv0 * r0 + bv1 * r1) : 0.f;
      const float sz = fmaxf(sz_raw, 0.f);
      float gsz = 0.f;
      constexpr int KA = K > 0 ? K : 1;   // array extent (the loop is empty for K = 0)
      float fr[3 * KA], wr[KA], gfr[3 * KA], gwr[KA];
      load_row<STORAGE, 3 * K>(V.freqs, k, fr);
      if (zatt) load_row<STORAGE, K>(V.weights, k, wr);
#pragma unroll
      for (int i = 0; i < K; ++i) {
        const float f0 = fr[3 * i], f1 = fr[3 * i + 1], f2 = fr[3 * i + 2];
        const float g0 = W[0] * f0 + W[1] * f1 + W[2] * f2;
        const float g1 = W[3] * f0 + W[4] * f1 + W[5] * f2;
        const float gg2 = W[6] * f0 + W[7] * f1 + W[8] * f2;
        const float fpz = gg2 + ux * g0 + uy * g1;
        const float gfx = g2[9 + 2 * i], gfy = g2[9 + 2 * i + 1];
        float gpz = r0 * gfx + r1 * gfy;
        const float Gi = g2[9 + 2 * K + i];
        const float c2 = zatt ? expf(-2.f * PI_SQ * fpz * fpz * sz) : 1.f;
        gwr[i] = c2 * Gi - G0;
        if (zatt) {
          const float garg = Gi * wr[i] * c2;              // dL/d(-2 pi^2 fpz^2 sz)
          gpz += garg * (-4.f * PI_SQ * fpz * sz);
          gsz += garg * (-2.f * PI_SQ * fpz * fpz);
        }
        gr0 += fpz * gfx;
        gr1 += fpz * gfy;
        const float gg0 = gfx * tzfx + gpz * ux;
        const float gg1 = gfy * tzfy + gpz * uy;
        const float ggz = gpz;
        gtz += gfx * g0 * ifx + gfy * g1 * ify;
        gux += gpz * g0;
        guy += gpz * g1;
        gfr[3 * i] = W[0] * gg0 + W[3] * gg1 + W[6] * ggz;
        gfr[3 * i + 1] = W[1] * gg0 + W[4] * gg1 + W[7] * ggz;
        gfr[3 * i + 2] = W[2] * gg0 + W[5] * gg1 + W[8] * ggz;
      }
      if (G.freqs) store_row<3 * K>(G.freqs, k, gfr);
      if (G.weights) store_row<K>(G.weights, k, gwr);
      // r = A^-1 b: gb = A^-1 gr, gA = -gb r^T (A symmetric, off-diagonal counted twice)
      const float u0 = iA00 * gr0 + iA01 * gr1, u1 = iA01 * gr0 + iA11 * gr1;
      gb0 = u0; gb1 = u1;
      gA00 -= u0 * r0;
      gA11 -= u1 * r1;
      gA01 -= u0 * r1 + u1 * r0;
      // sz = c - b^T A^-1 b: d/dc = 1, d/db = -2 r, d/dA = r r^T
      if (zatt && sz_raw > 0.f) {
        gcz = gsz;
        gb0 -= 2.f * r0 * gsz;
        gb1 -= 2.f * r1 * gsz;
        gA00 += r0 * r0 * gsz;
        gA11 += r1 * r1 * gsz;
        gA01 += 2.f * r0 * r1 * gsz;
      }
    }
    // ---- A = T Sigma T^T, b = T Sigma w3 ----
    float gS[9];
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j)
        gS[3 * i + j] = gA00 * T0[i] * T0[j] + gA01 * T0[i] * T1[j] + gA11 * T1[i] * T1[j] +
                        (gb0 * T0[i] + gb1 * T1[i]) * w3[j] + gcz * w3[i] * w3[j];
    float gT0[3], gT1[3];
    for (int j = 0; j < 3; ++j) {
      gT0[j] = 2.f * gA00 * U0[j] + gA01 * U1[j] + gb0 * Sw[j];
      gT1[j] = 2.f * gA11 * U1[j] + gA01 * U0[j] + gb1 * Sw[j];
    }
    // ---- T = J[0:2] W ----
    const float gJ00 = gT0[0] * W[0] + gT0[1] * W[1] + gT0[2] * W[2];
    const float gJ02 = gT0[0] * W[6] + gT0[1] * W[7] + gT0[2] * W[8];
    const float gJ11 = gT1[0] * W[3] + gT1[1] * W[4] + gT1[2] * W[5];
    const float gJ12 = gT1[0] * W[6] + gT1[1] * W[7] + gT1[2] * W[8];
    const float itz = 1.f / tz, itz2 = itz * itz;
    gtz += -V.fx * itz2 * gJ00 + V.fx * ux * itz2 * gJ02 - V.fy * itz2 * gJ11 + V.fy * uy * itz2 * gJ12;
    gux += -V.fx * itz * gJ02;
    guy += -V.fy * itz * gJ12;
    if (!clx) { gtx += gux * itz; gtz -= gux * tx * itz2; }
    if (!cly) { gty += guy * itz; gtz -= guy * ty * itz2; }
    // ---- projected mean ----
    gtx += g2[0] * V.fx * itz;
    gtz -= g2[0] * V.fx * tx * itz2;
    gty += g2[1] * V.fy * itz;
    gtz -= g2[1] * V.fy * ty * itz2;
    gmean[0] = W[0] * gtx + W[3] * gty + W[6] * gtz;
    gmean[1] = W[1] * gtx + W[4] * gty + W[7] * gtz;
    gmean[2] = W[2] * gtx + W[5] * gty + W[8] * gtz;
    // ---- Sigma = M M^T, M = R diag(s) ----
    float gM[9];
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) {
        float acc = 0.f;
        for (int l = 0; l < 3; ++l) acc += (gS[3 * i + l] + gS[3 * l + i]) * M[3 * l + j];
        gM[3 * i + j] = acc;
      }
    float gR[9];
    for (int j = 0; j < 3; ++j) {
      gscale[j] = gM[j] * R[j] + gM[3 + j] * R[3 + j] + gM[6 + j] * R[6 + j];
      for (int i = 0; i < 3; ++i) gR[3 * i + j] = gM[3 * i + j] * s[j];
    }
    const float gqw = 2.f * (-qz * gR[1] + qy * gR[2] + qz * gR[3] - qx * gR[5] - qy * gR[6] + qx * gR[7]);
    const float gqx = 2.f * (qy * gR[1] + qz * gR[2] + qy * gR[3] - 2.f * qx * gR[4] - qw * gR[5] + qz * gR[6] +
                             qw * gR[7] - 2.f * qx * gR[8]);
    const float gqy = 2.f * (-2.f * qy * gR[0] + qx * gR[1] + qw * gR[2] + qx * gR[3] + qz * gR[5] - qw * gR[6] +
                             qz * gR[7] - 2.f * qy * gR[8]);
    const float gqz = 2.f * (-2.f * qz * gR[0] - qw * gR[1] + qx * gR[2] + qw * gR[3] - 2.f * qz * gR[4] + qy * gR[5] +
                             qx * gR[6] + qy * gR[7]);
    const float dotq = qw * gqw + qx * gqx + qy * gqy + qz * gqz;
    gquat[0] = (gqw - qw * dotq) * iqn;
    gquat[1] = (gqx - qx * dotq) * iqn;
    gquat[2] = (gqy - qy * dotq) * iqn;
    gquat[3] = (gqz - qz * dotq) * iqn;
    // ---- SH colour ----
    {
      float dx = mx - V.campos[0], dy = my - V.campos[1], dz = mz - V.campos[2];
      const float len = sqrtf(dx * dx + dy * dy + dz * dz);
      const float il = 1.f / len;
      dx *= il; dy *= il; dz *= il;
      float Y[16];
      sh_eval(deg, dx, dy, dz, Y);
      const size_t shb = (size_t)k * nsh * 3;
      float raw[3] = {0.5f, 0.5f, 0.5f};
      float cw[16];
      float shc[48];
      load_sh_row<STORAGE>(V.sh, k, nsh, shc);
#pragma unroll
      for (int j = 0; j < 16; ++j)
        if (j < nsh)
#pragma unroll
          for (int c = 0; c < 3; ++c) raw[c] += Y[j] * shc[3 * j + c];
      float graw[3];
#pragma unroll
      for (int c = 0; c < 3; ++c) graw[c] = raw[c] < 0.f ? 0.f : g2[6 + c];
#pragma unroll
      for (int j = 0; j < 16; ++j)
        cw[j] = j < nsh ? shc[3 * j] * graw[0] + shc[3 * j + 1] * graw[1] + shc[3 * j + 2] * graw[2] : 0.f;
      if (G.sh) {
        if (nsh == 16 && (reinterpret_cast<uintptr_t>(G.sh) & 15) == 0) {
          float4* dst = reinterpret_cast<float4*>(G.sh + shb);
#pragma unroll
          for (int i = 0; i < 12; ++i) {
            float v[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) v[e] = Y[(4 * i + e) / 3] * graw[(4 * i + e) % 3];
            dst[i] = make_float4(v[0], v[1], v[2], v[3]);
          }
        } else {
#pragma unroll
          for (int j = 0; j < 16; ++j)
            if (j < nsh)
#pragma unroll
              for (int c = 0; c < 3; ++c) G.sh[shb + 3 * j + c] = Y[j] * graw[c];
        }
      }
      float gdx, gdy, gdz;
      sh_grad(deg, dx, dy, dz, cw, gdx, gdy, gdz);
      const float dd = dx * gdx + dy * gdy + dz * gdz;
      gmean[0] += (gdx - dx * dd) * il;
      gmean[1] += (gdy - dy * dd) * il;
      gmean[2] += (gdz - dz * dd) * il;
    }
    if (G.means) for (int i = 0; i < 3; ++i) G.means[3 * (size_t)k + i] = gmean[i];
    if (G.scales) for (int i = 0; i < 3; ++i) G.scales[3 * (size_t)k + i] = gscale[i];
    if (G.quats) store_row<4>(G.quats, k, gquat);
  }
}

// ------------------------------------------------------------------------------------------
// Host launchers
// ------------------------------------------------------------------------------------------
const void* setup_kernel_fn() { return reinterpret_cast<const void*>(k_setup); }

int device_sm_count() {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms > 0 ? sms : 1;
}

template <typename Kern>
static int persistent_grid(Kern kern, int threads, size_t smem, int sms) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem) != cudaSuccess || per_sm < 1) per_sm = 1;
  return per_sm * sms;
}

cudaError_t launch_setup(const FrameTable& tbl, const WsPtrs& p, const Launch& L) {
  launch_pdl<PDL_BIN>(k_setup, 1, 256, 0, L.stream, tbl, p);
  return cudaGetLastError();
}

template <int K, int ST>
static cudaError_t launch_pre_t(const FrameTable& tbl, const WsPtrs& p, const Launch& L) {
  static int bgrid = 0, egrid = 0, rgrid = 0;
  if (!bgrid) bgrid = persistent_grid(k_bin, BLOCK, 0, L.sm_count);
  if (!egrid) egrid = persistent_grid(k_emit, BLOCK, 0, L.sm_count);
  if (!rgrid) rgrid = persistent_grid(k_records<K, ST>, BLOCK, 0, L.sm_count);
  const int need = (int)((tbl.launch_prims + BLOCK - 1) / BLOCK);
  const int schunks = (int)((tbl.launch_prims + SCAN_CHUNK - 1) / SCAN_CHUNK);
  auto clampg = [](int g, int cap) { return g < 1 ? 1 : (g > cap ? cap : g); };
  launch_pdl<PDL_BIN>(k_bin, clampg(need, bgrid), BLOCK, 0, L.stream, p);
  const int sg = schunks < 1 ? 1 : schunks;   // one CTA per chunk (CTAs past the data return)
  launch_pdl<PDL_BIN>(k_scan_active, sg, BLOCK, 0, L.stream, p);
  cudaError_t e = launch_depth_sort(tbl, p, L);
  if (e != cudaSuccess) return e;
  launch_pdl<PDL_RANK>(k_scan_ranked, sg, BLOCK, 0, L.stream, p);
  launch_pdl<PDL_EMIT>(k_emit, clampg(need, egrid), BLOCK, 0, L.stream, p);
  launch_pdl<PDL_EMIT>(k_records<K, ST>, clampg(need, rgrid), BLOCK, 0, L.stream, p);
  return cudaGetLastError();
}

template <int K, int ST>
static cudaError_t launch_pre_bwd_t(const FrameTable& tbl, const WsPtrs& p, const gs_prim_grads& g, bool prezeroed,
                                    const Launch& L) {
  static int grid = 0;
  if (!grid) grid = persistent_grid(k_preprocess_bwd<K, ST>, BLOCK, 0, L.sm_count);
  const int n = tbl.v[0].n;
  const int nsh = (tbl.sh_degree + 1) * (tbl.sh_degree + 1);
  if (!prezeroed) launch_pdl<PDL_PBWD>(k_zero_grads, L.sm_count * 4, 256, 0, L.stream, g, n, K, nsh);
  int blocks = (n + BLOCK - 1) / BLOCK;
  if (blocks > grid) blocks = grid;
  if (blocks < 1) blocks = 1;
  launch_pdl<PDL_PBWD>(k_preprocess_bwd<K, ST>, blocks, BLOCK, 0, L.stream, p, g);
  return cudaGetLastError();
}

#define GS_DISPATCH_K(K_, ST_, FN, ...)                                 \
  switch (K_) {                                                         \
    case 0: return ST_ ? FN<0, 1>(__VA_ARGS__) : FN<0, 0>(__VA_ARGS__); \
    case 1: return ST_ ? FN<1, 1>(__VA_ARGS__) : FN<1, 0>(__VA_ARGS__); \
    case 2: return ST_ ? FN<2, 1>(__VA_ARGS__) : FN<2, 0>(__VA_ARGS__); \
    case 3: return ST_ ? FN<3, 1>(__VA_ARGS__) : FN<3, 0>(__VA_ARGS__); \
    case 4: return ST_ ? FN<4, 1>(__VA_ARGS__) : FN<4, 0>(__VA_ARGS__); \
    case 5: return ST_ ? FN<5, 1>(__VA_ARGS__) : FN<5, 0>(__VA_ARGS__); \
    case 6: return ST_ ? FN<6, 1>(__VA_ARGS__) : FN<6, 0>(__VA_ARGS__); \
    case 7: return ST_ ? FN<7, 1>(__VA_ARGS__) : FN<7, 0>(__VA_ARGS__); \
    case 8: return ST_ ? FN<8, 1>(__VA_ARGS__) : FN<8, 0>(__VA_ARGS__); \
    default: return cudaErrorInvalidValue;                              \
  }

cudaError_t launch_preprocess(const FrameTable& tbl, const WsPtrs& p, const Launch& L) {
  GS_DISPATCH_K(tbl.K, tbl.storage, launch_pre_t, tbl, p, L)
}

cudaError_t launch_preprocess_bwd(const FrameTable& tbl, const WsPtrs& p, const gs_prim_grads& g, bool prezeroed,
                                  const Launch& L) {
  GS_DISPATCH_K(tbl.K, tbl.storage, launch_pre_bwd_t, tbl, p, g, prezeroed, L)
}

}  // namespace gs
