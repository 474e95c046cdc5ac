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
// Render: 32 x 32 output tiles, one CTA each.  The CTA turns the (at most 50)
// triangles under its tile into records in FP64: for the triangle's cell
// origin q0, p0 = A q0 + t split into an integer base and an FP32 fraction.
// Each pixel then needs only small-magnitude FP32 arithmetic,
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
constexpr double kDetEps = 1e-9;
constexpr int kTile = 32;
constexpr int kMinCell = 8;
constexpr int kMaxRecCells = kTile / kMinCell + 1;  // cells per tile side

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
      for (int v = 0; v < kFitThreads / 32; ++v) s += sh[v][k];
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

__global__ void __launch_bounds__(kFitThreads) fit_groups_kernel(const float* q, const float* p, const float* w,
                                                                 const int64_t* offsets, double* theta,
                                                                 int32_t* status) {
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
  block_sum(m, sh);
  if (threadIdx.x == 0) {
    double th[6];
    int st = solve_affine(m, cy, cx, th);
    if (st != SWIFT_FIT_OK) write_identity(th);
    for (int k = 0; k < 6; ++k) theta[6 * g + k] = th[k];
    status[g] = st;
  }
}

__global__ void __launch_bounds__(kFitThreads) mesh_fit_kernel(const float* q, const float* p, const float* w,
                                                               int64_t n, swift_mesh mesh, int32_t band,
                                                               double* theta, int32_t* status) {
  __shared__ double sh[kFitThreads / 32][12];
  __shared__ int st_sh;
  const int t = blockIdx.x;
  const int c = t >> 1, half = t & 1;
  const int cy = c / mesh.nx, cx = c % mesh.nx;
  const double y0 = static_cast<double>(mesh.origin_y) + static_cast<double>(cy) * mesh.cell;
  const double x0 = static_cast<double>(mesh.origin_x) + static_cast<double>(cx) * mesh.cell;
  const double lo = -static_cast<double>(band), hi = static_cast<double>(mesh.cell) + band, dg = -2.0 * band;
  Moments m;
  m.zero();
  for (int64_t i = threadIdx.x; i < n; i += kFitThreads) {
    const double wi = w[i];
    if (!(wi > 0.0)) continue;
    const double dy = static_cast<double>(q[2 * i]) - y0, dx = static_cast<double>(q[2 * i + 1]) - x0;
    const bool box = dy >= lo && dy <= hi && dx >= lo && dx <= hi;
    const bool diag = half == 0 ? (dx - dy >= dg) : (dy - dx >= dg);
    if (box && diag) m.add(wi, dy, dx, static_cast<double>(p[2 * i]) - y0, static_cast<double>(p[2 * i + 1]) - x0);
  }
  block_sum(m, sh);
  double th[6];
  if (threadIdx.x == 0) st_sh = solve_affine(m, y0, x0, th);
  __syncthreads();
  if (st_sh != SWIFT_FIT_OK) {  // whole-point-set affine, centred on the mesh centre
    const double gy = mesh.origin_y + 0.5 * mesh.cell * mesh.ny, gx = mesh.origin_x + 0.5 * mesh.cell * mesh.nx;
    m.zero();
    for (int64_t i = threadIdx.x; i < n; i += kFitThreads) {
      const double wi = w[i];
      if (wi > 0.0)
        m.add(wi, static_cast<double>(q[2 * i]) - gy, static_cast<double>(q[2 * i + 1]) - gx,
              static_cast<double>(p[2 * i]) - gy, static_cast<double>(p[2 * i + 1]) - gx);
    }
    block_sum(m, sh);
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

struct RenderRec {
  float a_yy, a_yx, a_xy, a_xx;  // A
  float fy, fx;                  // fraction of p0 = A q0 + t
  int by, bx;                    // integer part of p0
};

template <typename TIn>
__device__ __forceinline__ float src_px(const TIn* s, long long pitch, int y, int x) {
  return static_cast<float>(s[static_cast<long long>(y) * pitch + x]);
}

template <typename TIn>
__global__ void __launch_bounds__(256) render_kernel(const TIn* src, long long src_pitch, int src_h, int src_w,
                                                     const double* theta, swift_mesh mesh, float* out,
                                                     long long out_pitch, int out_h, int out_w, float fill) {
  __shared__ RenderRec rec[kMaxRecCells * kMaxRecCells * 2];
  const int ty0 = blockIdx.y * kTile, tx0 = blockIdx.x * kTile;
  // cell of an output coordinate: floor division in integers, clamped to the mesh
  auto cell_i = [&](int v, int o, int n) {
    int d = v - o;
    int c = d >= 0 ? d / mesh.cell : -((-d + mesh.cell - 1) / mesh.cell);
    return c < 0 ? 0 : (c >= n ? n - 1 : c);
  };
  const int cy_lo = cell_i(ty0, mesh.origin_y, mesh.ny), cy_hi = cell_i(ty0 + kTile - 1, mesh.origin_y, mesh.ny);
  const int cx_lo = cell_i(tx0, mesh.origin_x, mesh.nx), cx_hi = cell_i(tx0 + kTile - 1, mesh.origin_x, mesh.nx);
  const int ncx = cx_hi - cx_lo + 1;
  const int nrec = (cy_hi - cy_lo + 1) * ncx * 2;
  for (int r = threadIdx.x; r < nrec; r += 256) {
    const int half = r & 1, cl = r >> 1;
    const int cy = cy_lo + cl / ncx, cx = cx_lo + cl % ncx;
    const double* th = theta + 6 * (2 * (cy * mesh.nx + cx) + half);
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
    rec[r] = R;
  }
  __syncthreads();
  const int tx = threadIdx.x & 31, tyl = threadIdx.x >> 5;
  const int x = tx0 + tx;
  if (x >= out_w) return;
  const int cx = cell_i(x, mesh.origin_x, mesh.nx);
  const int dxc = x - (mesh.origin_x + cx * mesh.cell);
#pragma unroll
  for (int k = 0; k < kTile / 8; ++k) {
    const int y = ty0 + tyl + 8 * k;
    if (y >= out_h) break;
    const int cy = cell_i(y, mesh.origin_y, mesh.ny);
    const int dyc = y - (mesh.origin_y + cy * mesh.cell);
    const int half = dxc >= dyc ? 0 : 1;
    const RenderRec R = rec[((cy - cy_lo) * ncx + (cx - cx_lo)) * 2 + half];
    const float fdy = static_cast<float>(dyc), fdx = static_cast<float>(dxc);
    const float ly = fmaf(R.a_yx, fdx, fmaf(R.a_yy, fdy, R.fy));
    const float lx = fmaf(R.a_xx, fdx, fmaf(R.a_xy, fdy, R.fx));
    const float fly = floorf(ly), flx = floorf(lx);
    long long iy = static_cast<long long>(R.by) + static_cast<long long>(fly);
    long long ix = static_cast<long long>(R.bx) + static_cast<long long>(flx);
    float fy = ly - fly, fx = lx - flx;
    // inside [0, h-1] x [0, w-1]
    const bool inside = iy >= 0 && ix >= 0 && (iy < src_h - 1 || (iy == src_h - 1 && fy == 0.f)) &&
                        (ix < src_w - 1 || (ix == src_w - 1 && fx == 0.f));
    float v = fill;
    if (inside) {
      if (iy == src_h - 1) {
        iy -= 1;
        fy = 1.f;
      }
      if (ix == src_w - 1) {
        ix -= 1;
        fx = 1.f;
      }
      const int yi = static_cast<int>(iy), xi = static_cast<int>(ix);
      const float s00 = src_px(src, src_pitch, yi, xi), s01 = src_px(src, src_pitch, yi, xi + 1);
      const float s10 = src_px(src, src_pitch, yi + 1, xi), s11 = src_px(src, src_pitch, yi + 1, xi + 1);
      const float top = fmaf(fx, s01 - s00, s00), bot = fmaf(fx, s11 - s10, s10);
      v = fmaf(fy, bot - top, top);
    }
    out[static_cast<long long>(y) * out_pitch + x] = v;
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

extern "C" swift_status swift_fit_affine(const float* q, const float* p, const float* w, const int64_t* offsets,
                                         int32_t n_groups, double* theta, int32_t* status, void* stream) {
  if (n_groups < 0) return SWIFT_ERR_INVALID_ARG;
  if (n_groups == 0) return SWIFT_OK;
  if (!q || !p || !w || !offsets || !theta || !status) return SWIFT_ERR_INVALID_ARG;
  if (cudaGetLastError() != cudaSuccess) return SWIFT_ERR_CUDA;
  swift::fit_groups_kernel<<<n_groups, swift::kFitThreads, 0, static_cast<cudaStream_t>(stream)>>>(q, p, w, offsets,
                                                                                                     theta, status);
  return cudaGetLastError() == cudaSuccess ? SWIFT_OK : SWIFT_ERR_CUDA;
}

extern "C" swift_status swift_mesh_fit(const float* q, const float* p, const float* w, int64_t n_points,
                                       const swift_mesh* mesh, int32_t band, double* theta, int32_t* status,
                                       void* stream) {
  if (n_points < 0 || band < 0 || !swift::mesh_ok(mesh) || !theta || !status) return SWIFT_ERR_INVALID_ARG;
  if (n_points > 0 && (!q || !p || !w)) return SWIFT_ERR_INVALID_ARG;
  if (cudaGetLastError() != cudaSuccess) return SWIFT_ERR_CUDA;
  const long long T = 2ll * mesh->ny * mesh->nx;
  swift::mesh_fit_kernel<<<static_cast<unsigned>(T), swift::kFitThreads, 0, static_cast<cudaStream_t>(stream)>>>(
      q, p, w, n_points, *mesh, band, theta, status);
  return cudaGetLastError() == cudaSuccess ? SWIFT_OK : SWIFT_ERR_CUDA;
}

extern "C" swift_status swift_render(const swift_image* src, swift_dtype dtype, const double* theta,
                                     const swift_mesh* mesh, float* out, int32_t out_h, int32_t out_w,
                                     int64_t out_pitch, float fill, void* stream) {
  if (!src || !src->data || src->height < 2 || src->width < 2 || src->pitch < src->width) return SWIFT_ERR_INVALID_ARG;
  if (dtype != SWIFT_IN_U8 && dtype != SWIFT_IN_F32) return SWIFT_ERR_INVALID_ARG;
  if (!swift::mesh_ok(mesh) || !theta || !out || out_h < 0 || out_w < 0 || out_pitch < out_w) return SWIFT_ERR_INVALID_ARG;
  if (out_h == 0 || out_w == 0) return SWIFT_OK;
  if (cudaGetLastError() != cudaSuccess) return SWIFT_ERR_CUDA;
  const dim3 grid((out_w + swift::kTile - 1) / swift::kTile, (out_h + swift::kTile - 1) / swift::kTile);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (dtype == SWIFT_IN_U8)
    swift::render_kernel<uint8_t><<<grid, 256, 0, st>>>(static_cast<const uint8_t*>(src->data), src->pitch,
                                                          src->height, src->width, theta, *mesh, out, out_pitch,
                                                          out_h, out_w, fill);
  else
    swift::render_kernel<float><<<grid, 256, 0, st>>>(static_cast<const float*>(src->data), src->pitch, src->height,
                                                        src->width, theta, *mesh, out, out_pitch, out_h, out_w, fill);
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
