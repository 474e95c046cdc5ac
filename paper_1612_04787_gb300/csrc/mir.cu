// Rendering step ("mir", Sec. III module list; Sec. IV): weighted least-squares
// affines from swim correspondence points, a locally affine triangle mesh, and
// texture-mapped rendering of a section through the mesh.
//
// Correspondence i: q_i (output / reference frame, (y, x)), p_i (source
// section), weight w_i >= 0.  Affine p = A q + t stored as
// (a_yy, a_yx, t_y, a_xy, a_xx, t_x), FP64.
//
// Fits: one CTA per problem accumulates the 12 weighted sums of centred
// coordinates in FP64 (fixed point-to-thread map and reduction tree, so the
// result is deterministic), then one thread solves the centred normal
// equations A = Cpq Sqq^-1, t = p_bar - A q_bar.  A problem is degenerate when
// sum w = 0 or det(Sqq) <= 1e-9 (tr Sqq / 2)^2.
//
// Mesh: ny x nx square cells of side c from the integer origin; triangle
// 2 (cy nx + cx) + 0 holds (x - x0) >= (y - y0), + 1 holds (x - x0) <=
// (y - y0).  A point supports a triangle when it lies within Chebyshev
// distance b of it (the triangle grown by the square [-b, b]^2: a box test and
// a relaxed diagonal test, exact in FP64 for float32 inputs).  Triangles whose
// support is degenerate take the whole-point-set affine (FALLBACK), else the
// identity (DEGENERATE).
//
// Render: a prepare kernel turns each triangle's affine into a record in FP64
// (once per mesh: the FP64 unit of this GPU is slow): for the triangle's cell
// corner q0, p0 = A q0 + t split into an integer base and an FP32 fraction.
// The render kernel (32 x 32 output tiles, 256 threads) reads records through
// L1, and each pixel needs only small-magnitude FP32 arithmetic,
// p = base + (frac + A (q - q0)), so large section coordinates cost no
// accuracy.  Bilinear sampling as the oracle: samples outside
// [0, h-1] x [0, w-1] take the fill value; the last row / column interpolate
// from the cell before it.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "../../include/swift.h"
#include "swift_internal.h"

namespace swift {

namespace {

constexpr int kFitThreads = 256;
constexpr int kMeshFitThreads = 64;  // measured against 128 and 256: fewer threads, shorter FP64 reductions
constexpr double kDetEps = 1e-9;
constexpr int kMinCell = 8;

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// 12 weighted sums of centred coordinates u = q - c, v = p - c
struct Moments {
  double W, uy, ux, vy, vx, uyy, uyx, uxx, vyuy, vyux, vxuy, vxux;
  __device__ void zero() { W = uy = ux = vy = vx = uyy = uyx = uxx = vyuy = vyux = vxuy = vxux = 0.0; }
  __device__ void add(double w, double qy, double qx, double py, double px) {
    W += w;
    uy = fma(w, qy, uy);
    ux = fma(w, qx, ux);
    vy = fma(w, py, vy);
    vx = fma(w, px, vx);
    uyy = fma(w * qy, qy, uyy);
    uyx = fma(w * qy, qx, uyx);
    uxx = fma(w * qx, qx, uxx);
    vyuy = fma(w * py, qy, vyuy);
    vyux = fma(w * py, qx, vyux);
    vxuy = fma(w * px, qy, vxuy);
    vxux = fma(w * px, qx, vxux);
  }
  __device__ double* as_array() { return &W; }
};

// block-wide sum of the moments (deterministic tree); result valid in thread 0
template <int NT>
__device__ void block_sum(Moments& m, double (*sh)[12]) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double* a = m.as_array();
#pragma unroll
  for (int k = 0; k < 12; ++k) a[k] = warp_sum_d(a[k]);
  if (lane == 0)
#pragma unroll
    for (int k = 0; k < 12; ++k) sh[warp][k] = a[k];
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int k = 0; k < 12; ++k) {
      double s = 0.0;
      for (int v = 0; v < NT / 32; ++v) s += sh[v][k];
      a[k] = s;
    }
  }
  __syncthreads();
}

// solve the centred normal equations; (cy, cx) is the centre used for u, v
__device__ int solve_affine(const Moments& m, double cy, double cx, double* th) {
  if (!(m.W > 0.0)) return SWIFT_FIT_DEGENERATE;
  const double qby = m.uy / m.W, qbx = m.ux / m.W, pby = m.vy / m.W, pbx = m.vx / m.W;
  const double syy = m.uyy - m.W * qby * qby, syx = m.uyx - m.W * qby * qbx, sxx = m.uxx - m.W * qbx * qbx;
  const double cyy = m.vyuy - m.W * pby * qby, cyx = m.vyux - m.W * pby * qbx;
  const double cxy = m.vxuy - m.W * pbx * qby, cxx = m.vxux - m.W * pbx * qbx;
  const double det = syy * sxx - syx * syx;
  const double tr = syy + sxx;
  if (!(det > kDetEps * (0.5 * tr) * (0.5 * tr))) return SWIFT_FIT_DEGENERATE;
  const double iyy = sxx / det, iyx = -syx / det, ixx = syy / det;
  const double a_yy = cyy * iyy + cyx * iyx, a_yx = cyy * iyx + cyx * ixx;
  const double a_xy = cxy * iyy + cxx * iyx, a_xx = cxy * iyx + cxx * ixx;
  // centred: v = A u + tc, tc = p_bar - A q_bar; absolute: t = tc + c - A c
  const double tcy = pby - (a_yy * qby + a_yx * qbx), tcx = pbx - (a_xy * qby + a_xx * qbx);
  th[0] = a_yy;
  th[1] = a_yx;
  th[2] = tcy + cy - (a_yy * cy + a_yx * cx);
  th[3] = a_xy;
  th[4] = a_xx;
  th[5] = tcx + cx - (a_xy * cy + a_xx * cx);
  return SWIFT_FIT_OK;
}

__device__ void write_identity(double* th) {
  th[0] = 1.0, th[1] = 0.0, th[2] = 0.0, th[3] = 0.0, th[4] = 1.0, th[5] = 0.0;
}

// keep: a degenerate group leaves its theta as it was (an update of previous
// affines) instead of writing the identity
__global__ void __launch_bounds__(kFitThreads) fit_groups_kernel(const float* q, const float* p, const float* w,
                                                                 const int64_t* offsets, double* theta,
                                                                 int32_t* status, int keep) {
  __shared__ double sh[kFitThreads / 32][12];
  const int g = blockIdx.x;
  const int64_t b = offsets[g], e = offsets[g + 1];
  const double cy = e > b ? q[2 * b] : 0.0, cx = e > b ? q[2 * b + 1] : 0.0;
  Moments m;
  m.zero();
  for (int64_t i = b + threadIdx.x; i < e; i += kFitThreads) {
    const double wi = w[i];
    if (wi > 0.0) m.add(wi, q[2 * i] - cy, q[2 * i + 1] - cx, p[2 * i] - cy, p[2 * i + 1] - cx);
  }
  block_sum<kFitThreads>(m, sh);
  if (threadIdx.x == 0) {
    double th[6];
    int st = solve_affine(m, cy, cx, th);
    if (st != SWIFT_FIT_OK) write_identity(th);
    if (st == SWIFT_FIT_OK || !keep)
      for (int k = 0; k < 6; ++k) theta[6 * g + k] = th[k];
    status[g] = st;
  }
}

__global__ void __launch_bounds__(kMeshFitThreads) mesh_fit_kernel(const float* q, const float* p, const float* w,
                                                                   int64_t n, swift_mesh mesh, int32_t band,
                                                                   double* theta, int32_t* status) {
  __shared__ double sh[kMeshFitThreads / 32][12];
  __shared__ int st_sh;
  const int t = blockIdx.x;
  const int c = t >> 1, half = t & 1;
  const int cy = c / mesh.nx, cx = c % mesh.nx;
  const double y0 = static_cast<double>(mesh.origin_y) + static_cast<double>(cy) * mesh.cell;
  const double x0 = static_cast<double>(mesh.origin_x) + static_cast<double>(cx) * mesh.cell;
  const double lo = -static_cast<double>(band), hi = static_cast<double>(mesh.cell) + band, dg = -2.0 * band;
  Moments m;
  m.zero();
  // FP32 prefilter with a 1 px margin (never rejects a supporting point), then
  // the exact FP64 test on the few candidates
  const float y0f = static_cast<float>(y0), x0f = static_cast<float>(x0);
  const float lof = static_cast<float>(lo) - 1.f, hif = static_cast<float>(hi) + 1.f;
  for (int64_t i = threadIdx.x; i < n; i += kMeshFitThreads) {
    const float wf = w[i];
    if (!(wf > 0.f)) continue;
    const float qyf = q[2 * i], qxf = q[2 * i + 1];
    const float ey = qyf - y0f, ex = qxf - x0f;
    if (!(ey >= lof && ey <= hif && ex >= lof && ex <= hif)) continue;
    const double wi = wf;
    const double dy = static_cast<double>(qyf) - y0, dx = static_cast<double>(qxf) - x0;
    const bool box = dy >= lo && dy <= hi && dx >= lo && dx <= hi;
    const bool diag = half == 0 ? (dx - dy >= dg) : (dy - dx >= dg);
    if (box && diag) m.add(wi, dy, dx, static_cast<double>(p[2 * i]) - y0, static_cast<double>(p[2 * i + 1]) - x0);
  }
  block_sum<kMeshFitThreads>(m, sh);
  double th[6];
  if (threadIdx.x == 0) st_sh = solve_affine(m, y0, x0, th);
  __syncthreads();
  if (st_sh != SWIFT_FIT_OK) {  // whole-point-set affine, centred on the mesh centre
    const double gy = mesh.origin_y + 0.5 * mesh.cell * mesh.ny, gx = mesh.origin_x + 0.5 * mesh.cell * mesh.nx;
    m.zero();
    for (int64_t i = threadIdx.x; i < n; i += kMeshFitThreads) {
      const double wi = w[i];
      if (wi > 0.0)
        m.add(wi, static_cast<double>(q[2 * i]) - gy, static_cast<double>(q[2 * i + 1]) - gx,
              static_cast<double>(p[2 * i]) - gy, static_cast<double>(p[2 * i + 1]) - gx);
    }
    block_sum<kMeshFitThreads>(m, sh);
    if (threadIdx.x == 0) {
      st_sh = solve_affine(m, gy, gx, th) == SWIFT_FIT_OK ? SWIFT_FIT_FALLBACK : SWIFT_FIT_DEGENERATE;
      if (st_sh == SWIFT_FIT_DEGENERATE) write_identity(th);
    }
  }
  if (threadIdx.x == 0) {
    for (int k = 0; k < 6; ++k) theta[6 * t + k] = th[k];
    status[t] = st_sh;
  }
}

// per-triangle render record (32 bytes): A in FP32, and p0 = A q0 + t for the
// triangle's cell corner q0 split into an FP32 fraction and an integer base
struct __align__(16) RenderRec {
  float a_yy, a_yx, a_xy, a_xx;  // A
  float fy, fx;                  // fraction of p0
  int by, bx;                    // integer part of p0
};
static_assert(sizeof(RenderRec) == 32, "record layout");

// Per-pixel coordinate arithmetic avoids float <-> int conversions, floor and
// integer division: small integers become floats through the exponent trick,
// and floor comes from the 1.5 * 2^23 rounding trick.  (Source bytes use the
// plain uint8 -> float conversion, which measured ~3 % faster than building
// the float from the mantissa.)
// |v| < 2^22 (pixel offsets from their cell, bounded by the render size limits)
__device__ __forceinline__ float small_int_to_float(int v) {
  return __int_as_float(0x4B400000 + v) - 12582912.0f;
}
__device__ __forceinline__ float src_val(const uint8_t* s) { return static_cast<float>(__ldg(s)); }
__device__ __forceinline__ float src_val(const float* s) { return __ldg(s); }
// floor of v (|v| < 2^22) as an integer and the fraction v - floor(v) in [0, 1)
__device__ __forceinline__ int floor_frac(float v, float& frac) {
  const float r = v + 12582912.0f;  // 1.5 * 2^23: r's low mantissa bits hold round(v)
  int ri = __float_as_int(r) - 0x4B400000;
  float rf = r - 12582912.0f;       // round(v), exactly
  if (rf > v) {
    ri -= 1;
    rf -= 1.0f;
  }
  frac = v - rf;
  return ri;
}

// one thread per triangle: the FP64 part of rendering, done once per mesh
__global__ void render_prepare_kernel(const double* theta, swift_mesh mesh, RenderRec* rec, int n_tri) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n_tri) return;
  const int c = t >> 1;
  const int cy = c / mesh.nx, cx = c % mesh.nx;
  const double* th = theta + 6 * t;
  const double q0y = static_cast<double>(mesh.origin_y) + static_cast<double>(cy) * mesh.cell;
  const double q0x = static_cast<double>(mesh.origin_x) + static_cast<double>(cx) * mesh.cell;
  const double p0y = th[0] * q0y + th[1] * q0x + th[2];
  const double p0x = th[3] * q0y + th[4] * q0x + th[5];
  const double by = floor(p0y), bx = floor(p0x);
  RenderRec R;
  R.a_yy = static_cast<float>(th[0]);
  R.a_yx = static_cast<float>(th[1]);
  R.a_xy = static_cast<float>(th[3]);
  R.a_xx = static_cast<float>(th[4]);
  R.fy = static_cast<float>(p0y - by);
  R.fx = static_cast<float>(p0x - bx);
  // bases far outside any section saturate (their pixels take the fill value)
  R.by = static_cast<int>(fmin(fmax(by, -1e9), 1e9));
  R.bx = static_cast<int>(fmin(fmax(bx, -1e9), 1e9));
  rec[t] = R;
}

// output value: float32 as is; uint8 rounded half to even and clamped to
// [0, 255] (the 1.5 * 2^23 rounding trick, no conversion instruction)
__device__ __forceinline__ void store_px(float* p, float v) { __stcs(p, v); }
__device__ __forceinline__ void store_px(uint8_t* p, float v) {
  const float c = fminf(fmaxf(v, 0.f), 255.f);  // NaN -> 0
  *p = static_cast<uint8_t>(__float_as_int(c + 12582912.0f) - 0x4B400000);
}

// IDX (below): int for images below 2^31 elements (cheaper address arithmetic), else long long
// Row-run form: a thread renders kRun adjacent pixels of one row (CTA tile
// kRunTileW x kRunTileH).  The cell and triangle walk advances one pixel at a
// time, the triangle's record is reloaded only when it changes, and the
// outputs leave in one vector store when the run is whole and aligned.  The
// per-pixel arithmetic: the sample point from the record (FP32 fraction of
// an integer base), floor and fraction, inside test with the last row and
// column inclusive, bilinear weights.
constexpr int kRun = 8;
constexpr int kRunTileW = 16 * kRun;  // 16 threads per row
constexpr int kRunTileH = 16;         // 256 threads

template <typename TOut>
__device__ __forceinline__ void store_run(TOut* p, const float (&v)[kRun]);
template <>
__device__ __forceinline__ void store_run<float>(float* p, const float (&v)[kRun]) {
  __stcs(reinterpret_cast<float4*>(p), make_float4(v[0], v[1], v[2], v[3]));
  __stcs(reinterpret_cast<float4*>(p) + 1, make_float4(v[4], v[5], v[6], v[7]));
}
template <>
__device__ __forceinline__ void store_run<uint8_t>(uint8_t* p, const float (&v)[kRun]) {
  uint32_t w[2] = {0u, 0u};
#pragma unroll
  for (int k = 0; k < kRun; ++k) {
    const float c = fminf(fmaxf(v[k], 0.f), 255.f);  // NaN -> 0; half-to-even rounding below
    w[k >> 2] |= static_cast<uint32_t>(__float_as_int(c + 12582912.0f) - 0x4B400000) << (8 * (k & 3));
  }
  *reinterpret_cast<uint2*>(p) = make_uint2(w[0], w[1]);
}

template <typename TIn, typename TOut, typename IDX>
__global__ void __launch_bounds__(256) render_run_kernel(const TIn* src, IDX src_pitch, int src_h, int src_w,
                                                         const RenderRec* rec, swift_mesh mesh, TOut* out,
                                                         IDX out_pitch, int out_h, int out_w, float fill,
                                                         int vec_out) {
  // row tiles on grid x (up to 2^20 / 16 of them), column tiles on grid y
  const int ty0 = blockIdx.x * kRunTileH, tx0 = blockIdx.y * kRunTileW;
  __shared__ int tile_cells[4];  // cy0, dy0, cx0, dx0 of the tile's first pixel
  if (threadIdx.x == 0) {
    auto cell_i = [&](int v, int o, int n) {
      const int d = v - o;
      const int c = d >= 0 ? d / mesh.cell : -((-d + mesh.cell - 1) / mesh.cell);
      return c < 0 ? 0 : (c >= n ? n - 1 : c);
    };
    const int cy0 = cell_i(ty0, mesh.origin_y, mesh.ny), cx0 = cell_i(tx0, mesh.origin_x, mesh.nx);
    tile_cells[0] = cy0;
    tile_cells[1] = ty0 - (mesh.origin_y + cy0 * mesh.cell);
    tile_cells[2] = cx0;
    tile_cells[3] = tx0 - (mesh.origin_x + cx0 * mesh.cell);
  }
  __syncthreads();
  const int tyl = threadIdx.x >> 4, txl = threadIdx.x & 15;
  const int y = ty0 + tyl, x0 = tx0 + kRun * txl;
  if (y >= out_h || x0 >= out_w) return;
  // cells advance while the offset reaches the cell side, and stay clamped
  // at the last cell (pixels beyond the mesh use the border cells)
  int cy = tile_cells[0], dyc = tile_cells[1] + tyl;
  while (dyc >= mesh.cell && cy < mesh.ny - 1) {
    dyc -= mesh.cell;
    cy += 1;
  }
  int cx = tile_cells[2], dxc = tile_cells[3] + kRun * txl;
  while (dxc >= mesh.cell && cx < mesh.nx - 1) {
    dxc -= mesh.cell;
    cx += 1;
  }
  const float fdy = small_int_to_float(dyc);
  const float cellf = small_int_to_float(mesh.cell);
  float fdx = small_int_to_float(dxc);
  // phase 1: the triangle walk and the sample points of the run
  int yi[kRun], xi[kRun];
  float fyv[kRun], fxv[kRun];
  bool ins[kRun];
  int cur = -1;
  float4 r0 = make_float4(0.f, 0.f, 0.f, 0.f), r1 = r0;
#pragma unroll
  for (int k = 0; k < kRun; ++k) {
    if (k > 0) {
      dxc += 1;
      fdx += 1.0f;
      if (dxc >= mesh.cell && cx < mesh.nx - 1) {
        cx += 1;
        dxc -= mesh.cell;
        fdx -= cellf;
      }
    }
    const int idx = 2 * (cy * mesh.nx + cx) + (dxc >= dyc ? 0 : 1);
    if (idx != cur) {
      const float4* rp = reinterpret_cast<const float4*>(rec + idx);
      r0 = __ldg(rp);      // (a_yy, a_yx, a_xy, a_xx)
      r1 = __ldg(rp + 1);  // (fy, fx, by, bx)
      cur = idx;
    }
    const float sy = fmaf(r0.y, fdx, fmaf(r0.x, fdy, r1.x));  // local sample point
    const float sx = fmaf(r0.w, fdx, fmaf(r0.z, fdy, r1.y));
    const float ly = fminf(fmaxf(sy, -4e6f), 4e6f);  // |sum with the base| < 2^31; NaN -> outside
    const float lx = fminf(fmaxf(sx, -4e6f), 4e6f);
    float fy, fx;
    int iy = __float_as_int(r1.z) + floor_frac(ly, fy);
    int ix = __float_as_int(r1.w) + floor_frac(lx, fx);
    const bool inside = iy >= 0 && ix >= 0 && (iy < src_h - 1 || (iy == src_h - 1 && fy == 0.f)) &&
                        (ix < src_w - 1 || (ix == src_w - 1 && fx == 0.f));
    if (iy == src_h - 1) {
      iy -= 1;
      fy = 1.f;
    }
    if (ix == src_w - 1) {
      ix -= 1;
      fx = 1.f;
    }
    ins[k] = inside;
    yi[k] = inside ? iy : 0;  // outside pixels read the (valid) corner and take the fill value
    xi[k] = inside ? ix : 0;
    fyv[k] = fy;
    fxv[k] = fx;
  }
  // phase 2: every source load of the run in flight together; phase 3: interpolate
  float v[kRun];
#pragma unroll
  for (int k = 0; k < kRun; ++k) {
    const TIn* s0 = src + (static_cast<IDX>(yi[k]) * src_pitch + xi[k]);
    const float a = src_val(s0), b = src_val(s0 + 1), c = src_val(s0 + src_pitch), d = src_val(s0 + src_pitch + 1);
    const float top = fmaf(fxv[k], b - a, a);
    const float bot = fmaf(fxv[k], d - c, c);
    v[k] = ins[k] ? fmaf(fyv[k], bot - top, top) : fill;
  }
  TOut* o = out + (static_cast<IDX>(y) * out_pitch + x0);
  if (vec_out && x0 + kRun <= out_w) {
    store_run<TOut>(o, v);
  } else {
#pragma unroll
    for (int k = 0; k < kRun; ++k)
      if (x0 + k < out_w) store_px(o + k, v[k]);
  }
}

// correspondences from swim results: q = reference window centre, p = moving
// window centre + subpixel shift, w = SNR of OK windows with a finite SNR at
// least min_snr, else 0
__global__ void correspondences_kernel(const swift_result* res, const int32_t* ref_origin, const int32_t* mov_origin,
                                       long long B, int n, float min_snr, float* q, float* p, float* w) {
  const long long b = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x;
  if (b >= B) return;
  const swift_result r = res[b];
  const float c = 0.5f * n;
  q[2 * b] = ref_origin[2 * b] + c;
  q[2 * b + 1] = ref_origin[2 * b + 1] + c;
  const bool ok = r.status == SWIFT_WIN_OK && r.snr <= 3.4e38f && r.snr >= min_snr;
  p[2 * b] = mov_origin[2 * b] + c + (ok ? r.sy : 0.f);
  p[2 * b + 1] = mov_origin[2 * b + 1] + c + (ok ? r.sx : 0.f);
  w[b] = ok ? r.snr : 0.f;
}

bool mesh_ok(const swift_mesh* m) {
  return m && m->cell >= kMinCell && m->ny >= 1 && m->nx >= 1 &&
         static_cast<long long>(m->ny) * m->nx <= (1ll << 24) &&
         llabs(static_cast<long long>(m->origin_y)) < (1ll << 28) && llabs(static_cast<long long>(m->origin_x)) < (1ll << 28) &&
         static_cast<long long>(m->cell) * (m->ny > m->nx ? m->ny : m->nx) < (1ll << 28);
}

}  // namespace

}  // namespace swift

namespace {
swift_status fit_affine_impl(const float* q, const float* p, const float* w, const int64_t* offsets,
                             int32_t n_groups, double* theta, int32_t* status, int keep, void* stream) {
  if (n_groups < 0) return SWIFT_ERR_INVALID_ARG;
  if (n_groups == 0) return SWIFT_OK;
  if (!q || !p || !w || !offsets || !theta || !status) return SWIFT_ERR_INVALID_ARG;
  if (cudaGetLastError() != cudaSuccess) return SWIFT_ERR_CUDA;
  swift::fit_groups_kernel<<<n_groups, swift::kFitThreads, 0, static_cast<cudaStream_t>(stream)>>>(
      q, p, w, offsets, theta, status, keep);
  return cudaGetLastError() == cudaSuccess ? SWIFT_OK : SWIFT_ERR_CUDA;
}
}  // namespace

extern "C" swift_status swift_fit_affine(const float* q, const float* p, const float* w, const int64_t* offsets,
                                         int32_t n_groups, double* theta, int32_t* status, void* stream) {
  return fit_affine_impl(q, p, w, offsets, n_groups, theta, status, 0, stream);
}

extern "C" swift_status swift_fit_affine_update(const float* q, const float* p, const float* w,
                                                const int64_t* offsets, int32_t n_groups, double* theta,
                                                int32_t* status, void* stream) {
  return fit_affine_impl(q, p, w, offsets, n_groups, theta, status, 1, stream);
}

extern "C" swift_status swift_mesh_fit(const float* q, const float* p, const float* w, int64_t n_points,
                                       const swift_mesh* mesh, int32_t band, double* theta, int32_t* status,
                                       void* stream) {
  if (n_points < 0 || band < 0 || !swift::mesh_ok(mesh) || !theta || !status) return SWIFT_ERR_INVALID_ARG;
  if (n_points > 0 && (!q || !p || !w)) return SWIFT_ERR_INVALID_ARG;
  if (cudaGetLastError() != cudaSuccess) return SWIFT_ERR_CUDA;
  const long long T = 2ll * mesh->ny * mesh->nx;
  swift::mesh_fit_kernel<<<static_cast<unsigned>(T), swift::kMeshFitThreads, 0,
                           static_cast<cudaStream_t>(stream)>>>(
      q, p, w, n_points, *mesh, band, theta, status);
  return cudaGetLastError() == cudaSuccess ? SWIFT_OK : SWIFT_ERR_CUDA;
}

extern "C" swift_status swift_render_prepare(const double* theta, const swift_mesh* mesh, void* records,
                                             void* stream) {
  if (!swift::mesh_ok(mesh) || !theta || !records || (reinterpret_cast<uintptr_t>(records) & 15) != 0)
    return SWIFT_ERR_INVALID_ARG;
  if (cudaGetLastError() != cudaSuccess) return SWIFT_ERR_CUDA;
  const int T = 2 * mesh->ny * mesh->nx;
  swift::render_prepare_kernel<<<(T + 255) / 256, 256, 0, static_cast<cudaStream_t>(stream)>>>(
      theta, *mesh, static_cast<swift::RenderRec*>(records), T);
  return cudaGetLastError() == cudaSuccess ? SWIFT_OK : SWIFT_ERR_CUDA;
}

namespace swift {
namespace {
template <typename TIn, typename TOut>
void launch_render(cudaStream_t st, bool small, const TIn* src, const swift_image* im, const RenderRec* rec,
                   const swift_mesh& mesh, TOut* out, int64_t out_pitch, int out_h, int out_w, float fill) {
  const dim3 grid((out_h + kRunTileH - 1) / kRunTileH, (out_w + kRunTileW - 1) / kRunTileW);
  // a run's vector store needs its first pixel aligned to the run's bytes
  constexpr uintptr_t kRunBytes = kRun * sizeof(TOut);
  const int vec_out = (reinterpret_cast<uintptr_t>(out) % (kRunBytes < 16 ? kRunBytes : 16) == 0 &&
                       (static_cast<uintptr_t>(out_pitch) * sizeof(TOut)) % (kRunBytes < 16 ? kRunBytes : 16) == 0)
                          ? 1
                          : 0;
  if (small)
    render_run_kernel<TIn, TOut, int><<<grid, 256, 0, st>>>(src, static_cast<int>(im->pitch), im->height, im->width,
                                                            rec, mesh, out, static_cast<int>(out_pitch), out_h, out_w,
                                                            fill, vec_out);
  else
    render_run_kernel<TIn, TOut, long long><<<grid, 256, 0, st>>>(src, im->pitch, im->height, im->width, rec, mesh,
                                                                  out, out_pitch, out_h, out_w, fill, vec_out);
}
}  // namespace
}  // namespace swift

extern "C" swift_status swift_render(const swift_image* src, swift_dtype dtype, const void* records,
                                     const swift_mesh* mesh, void* out, swift_dtype out_dtype, int32_t out_h,
                                     int32_t out_w, int64_t out_pitch, float fill, void* stream) {
  if (!src || !src->data || src->height < 2 || src->width < 2 || src->pitch < src->width) return SWIFT_ERR_INVALID_ARG;
  if (dtype != SWIFT_IN_U8 && dtype != SWIFT_IN_F32) return SWIFT_ERR_INVALID_ARG;
  if (out_dtype != SWIFT_IN_U8 && out_dtype != SWIFT_IN_F32) return SWIFT_ERR_INVALID_ARG;
  if (!swift::mesh_ok(mesh) || !records || (reinterpret_cast<uintptr_t>(records) & 15) != 0 || !out || out_h < 0 ||
      out_w < 0 || out_pitch < out_w)
    return SWIFT_ERR_INVALID_ARG;
  if (out_h == 0 || out_w == 0) return SWIFT_OK;
  // pixel offsets from their cell stay below 2^22 (small-integer float conversion)
  if (out_h > (1 << 20) || out_w > (1 << 20) || llabs(static_cast<long long>(mesh->origin_y)) > (1 << 20) ||
      llabs(static_cast<long long>(mesh->origin_x)) > (1 << 20) ||
      static_cast<long long>(mesh->cell) * (mesh->ny > mesh->nx ? mesh->ny : mesh->nx) > (1 << 20))
    return SWIFT_ERR_INVALID_ARG;
  if (cudaGetLastError() != cudaSuccess) return SWIFT_ERR_CUDA;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const swift::RenderRec* rec = static_cast<const swift::RenderRec*>(records);
  const bool small = static_cast<long long>(src->height) * src->pitch < (1ll << 31) &&
                     static_cast<long long>(out_h) * out_pitch < (1ll << 31);
  const uint8_t* s8 = static_cast<const uint8_t*>(src->data);
  const float* sf = static_cast<const float*>(src->data);
  float* of = static_cast<float*>(out);
  uint8_t* o8 = static_cast<uint8_t*>(out);
  if (dtype == SWIFT_IN_U8) {
    if (out_dtype == SWIFT_IN_F32)
      swift::launch_render(st, small, s8, src, rec, *mesh, of, out_pitch, out_h, out_w, fill);
    else
      swift::launch_render(st, small, s8, src, rec, *mesh, o8, out_pitch, out_h, out_w, fill);
  } else {
    if (out_dtype == SWIFT_IN_F32)
      swift::launch_render(st, small, sf, src, rec, *mesh, of, out_pitch, out_h, out_w, fill);
    else
      swift::launch_render(st, small, sf, src, rec, *mesh, o8, out_pitch, out_h, out_w, fill);
  }
  return cudaGetLastError() == cudaSuccess ? SWIFT_OK : SWIFT_ERR_CUDA;
}

extern "C" swift_status swift_correspondences(const swift_result* results, const int32_t* ref_origin,
                                              const int32_t* mov_origin, int64_t n_windows, int32_t n, float min_snr,
                                              float* q, float* p, float* w, void* stream) {
  if (n_windows < 0 || n < 1) return SWIFT_ERR_INVALID_ARG;
  if (n_windows == 0) return SWIFT_OK;
  if (!results || !ref_origin || !mov_origin || !q || !p || !w) return SWIFT_ERR_INVALID_ARG;
  if (cudaGetLastError() != cudaSuccess) return SWIFT_ERR_CUDA;
  const long long blocks = (n_windows + 255) / 256;
  if (blocks > 0x7fffffffll) return SWIFT_ERR_INVALID_ARG;
  swift::correspondences_kernel<<<static_cast<unsigned>(blocks), 256, 0, static_cast<cudaStream_t>(stream)>>>(
      results, ref_origin, mov_origin, n_windows, n, min_snr, q, p, w);
  return cudaGetLastError() == cudaSuccess ? SWIFT_OK : SWIFT_ERR_CUDA;
}
