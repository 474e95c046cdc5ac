// Fused forward matching kernel: one window pair per cluster of C CTAs.
//
// Per window pair (Sec. III, the swim step):
//   gather -> weighted-mean removal + cosine taper -> z = m' + i r'
//   -> 2D DFT of z (rows, then columns) -> unpack M, R from Z (Hermitian
//   split) -> C = M conj(R) -> G = C |C|^-w / n^2, G[0,0] = 0
//   -> inverse 2D DFT of the Hermitian G (columns for kx <= n/2 only, then
//   rows two at a time as one complex transform) -> real match response s
//   -> peak (argmax, smallest index on ties) -> SNR against the background
//   outside the exclusion disc -> separable parabola subpixel fit.
//
// Layout: the n x n complex field is split across the C CTAs of a cluster.
// In the row phase CTA r owns rows [r*n/C, (r+1)*n/C); in the column phase it
// owns n/C columns closed under kx -> -kx, so the Hermitian unpack stays
// local.  The two redistributions go through distributed shared memory:
// every thread first holds its share of the slab in registers, the cluster
// synchronises, and the values are stored straight into the owner CTA's
// shared memory (st.shared::cluster), followed by a second cluster barrier.
// With C = 1 the same code runs inside one CTA.
//
// Each 1D transform of length n = R1 * R2 is two Stockham radix passes done
// in registers (radix R1 on inputs j + (n/R1) m, radix R2 with twiddles
// W_n^{j m} on inputs j + R1 m), with shared memory between them; row lines
// are padded by one element every R1 to keep the strided stores free of bank
// conflicts.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "dft_regs.cuh"
#include "swift_internal.h"

namespace swift {

template <int N, int C>
struct Geometry;
template <>
struct Geometry<64, 1> {
  static constexpr int T = 256, R1 = 8, R2 = 8;
};
template <>
struct Geometry<128, 1> {
  static constexpr int T = 512, R1 = 16, R2 = 8;
};
template <>
struct Geometry<256, 4> {
  static constexpr int T = 512, R1 = 16, R2 = 16;
};

template <int N, int C>
struct Plan2D {
  using G = Geometry<N, C>;
  static constexpr int T = G::T, R1 = G::R1, R2 = G::R2;
  static constexpr int ROWS = N / C;      // lines owned per CTA in each phase
  static constexpr int Q = N / (2 * C);  // kx in [Q r, Q r + Q) plus their partners
  static constexpr int RS = N + N / R1;  // padded row stride (complex elements)
  static constexpr int HALF = ROWS / 2;  // packed inverse rows per CTA
  // tasks per thread in each pass
  static constexpr int KA = ROWS * (N / R1) / T;   // radix-R1 tasks, full slab
  static constexpr int KB = ROWS * (N / R2) / T;   // radix-R2 tasks, full slab
  static constexpr int KAh = HALF * (N / R1) / T;  // radix-R1 tasks, half slab
  static constexpr int KBh = HALF * (N / R2) / T;  // radix-R2 tasks, half slab
  static_assert(R1 * R2 == N, "radix split");
  static_assert(KA * T == ROWS * (N / R1) && KB * T == ROWS * (N / R2), "task split");
  static_assert(KAh * T == HALF * (N / R1) && KBh * T == HALF * (N / R2), "task split (half)");
  static_assert(KAh >= 1 && KBh >= 1, "at least one task per thread");
  static_assert((HALF % R1) == 0, "row pairing must stay inside one thread");
  // shared memory (complex elements)
  static constexpr int ROW_SLAB = ROWS * RS;
  static constexpr int COL_SLAB = N * ROWS;
  static constexpr int PACKED = HALF * RS;
  static constexpr int SURF = ROWS * N / 2;  // floats / 2
  static constexpr int SLAB = (ROW_SLAB > COL_SLAB ? (ROW_SLAB > PACKED + SURF ? ROW_SLAB : PACKED + SURF)
                                                   : (COL_SLAB > PACKED + SURF ? COL_SLAB : PACKED + SURF));
  // padded index within a row line
  static __device__ __forceinline__ int phys(int p) { return p + p / R1; }
  // column ownership: (rank, local column) -> kx, and kx -> (rank, local column)
  static __device__ __forceinline__ int kx_of(int r, int lc) {
    if (lc < Q) return Q * r + lc;
    if (r == 0 && lc == Q) return N / 2;
    return N - (Q * r + lc - Q);
  }
  static __device__ __forceinline__ void owner_of(int kx, int& r, int& lc) {
    if (kx < N / 2) {
      r = kx / Q;
      lc = kx % Q;
    } else if (kx == N / 2) {
      r = 0;
      lc = Q;
    } else {
      int k2 = N - kx;
      r = k2 / Q;
      lc = Q + k2 % Q;
    }
  }
};

// ---------------------------------------------------------------------------
// cluster helpers (C == 1: plain shared memory and __syncthreads)
// ---------------------------------------------------------------------------
template <int C>
__device__ __forceinline__ unsigned cluster_rank() {
  if constexpr (C == 1) {
    return 0;
  } else {
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
  }
}

template <int C>
__device__ __forceinline__ void cluster_barrier() {
  if constexpr (C == 1) {
    __syncthreads();
  } else {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
  }
}

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// shared::cluster address of the same offset in CTA `rank`
template <int C>
__device__ __forceinline__ uint32_t map_rank(uint32_t local, unsigned rank) {
  if constexpr (C == 1) {
    return local;
  } else {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(local), "r"(rank));
    return r;
  }
}

template <int C>
__device__ __forceinline__ void st_remote(uint32_t addr, float2 v) {
  if constexpr (C == 1) {
    asm volatile("st.shared.v2.f32 [%0], {%1, %2};" ::"r"(addr), "f"(v.x), "f"(v.y) : "memory");
  } else {
    asm volatile("st.shared::cluster.v2.f32 [%0], {%1, %2};" ::"r"(addr), "f"(v.x), "f"(v.y) : "memory");
  }
}

template <int C>
__device__ __forceinline__ void st_remote_f64(uint32_t addr, double v) {
  if constexpr (C == 1) {
    asm volatile("st.shared.f64 [%0], %1;" ::"r"(addr), "d"(v) : "memory");
  } else {
    asm volatile("st.shared::cluster.f64 [%0], %1;" ::"r"(addr), "d"(v) : "memory");
  }
}

template <int C>
__device__ __forceinline__ void st_remote_u64(uint32_t addr, unsigned long long v) {
  if constexpr (C == 1) {
    asm volatile("st.shared.u64 [%0], %1;" ::"r"(addr), "l"(v) : "memory");
  } else {
    asm volatile("st.shared::cluster.u64 [%0], %1;" ::"r"(addr), "l"(v) : "memory");
  }
}

// ---------------------------------------------------------------------------
// reductions
// ---------------------------------------------------------------------------
// (value, index) ordering for the argmax: larger value wins, then smaller index.
// Packed so that a single unsigned 64-bit max gives the winner: the high 32
// bits hold an order-preserving encoding of the float, the low 32 bits hold
// ~index.
__device__ __forceinline__ unsigned long long argmax_key(float v, uint32_t idx) {
  uint32_t b = __float_as_uint(v);
  b = (b & 0x80000000u) ? ~b : (b | 0x80000000u);
  return (static_cast<unsigned long long>(b) << 32) | static_cast<unsigned long long>(~idx);
}
__device__ __forceinline__ float key_value(unsigned long long k) {
  uint32_t b = static_cast<uint32_t>(k >> 32);
  b = (b & 0x80000000u) ? (b & 0x7fffffffu) : ~b;
  return __uint_as_float(b);
}
__device__ __forceinline__ uint32_t key_index(unsigned long long k) { return ~static_cast<uint32_t>(k); }

__device__ __forceinline__ unsigned long long warp_max_u64(unsigned long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    unsigned long long w = __shfl_xor_sync(0xffffffffu, v, o);
    v = w > v ? w : v;
  }
  return v;
}
__device__ __forceinline__ double warp_sum_f64(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ float warp_sum_f32(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ float warp_min_f32(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fminf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
__device__ __forceinline__ float warp_max_f32(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// ---------------------------------------------------------------------------
// the kernel's shared-memory scratch (besides the slab)
// ---------------------------------------------------------------------------
constexpr int kMaxC = 4;
struct __align__(16) Scratch {
  // per-warp partials (filled by each CTA for its own block reduction)
  double wsum[32][2];
  float wmin[32][2], wmax[32][2];
  int wbad[32];
  unsigned long long wkey[32];
  double wbg[32][3];
  // cluster all-gather slots: written by every CTA into every CTA
  double csum[kMaxC][2];
  float cmin[kMaxC][2], cmax[kMaxC][2];
  int cbad[kMaxC];
  unsigned long long ckey[kMaxC];
  double cbg[kMaxC][3];
  float nb[4];  // peak neighbours for the subpixel fit: y-1, y+1, x-1, x+1 (rank 0)
  double stat[2];
  float peak_val;
  int peak_idx;
  int status;
};

// ---------------------------------------------------------------------------
// input element loads
// ---------------------------------------------------------------------------
template <typename TIn>
__device__ __forceinline__ float load_px(const TIn* p) {
  if constexpr (sizeof(TIn) == 1) {
    return static_cast<float>(__ldg(reinterpret_cast<const unsigned char*>(p)));
  } else {
    return __ldg(reinterpret_cast<const float*>(p));
  }
}

// ---------------------------------------------------------------------------
// the fused forward kernel
// ---------------------------------------------------------------------------
template <int N, int C, typename TIn>
__global__ void __launch_bounds__(Plan2D<N, C>::T, 1) swim_forward_kernel(const MatchLaunch L) {
  using P = Plan2D<N, C>;
  constexpr int T = P::T, R1 = P::R1, R2 = P::R2, ROWS = P::ROWS, Q = P::Q, RS = P::RS;
  constexpr int NW = T / 32;

  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* slab = reinterpret_cast<float2*>(smem_raw);
  float2* twid = slab + P::SLAB;                             // [R2][R1] W_N^{j m}
  float* taper = reinterpret_cast<float*>(twid + N);         // [N]
  Scratch* sc = reinterpret_cast<Scratch*>(taper + N);

  const int tid = threadIdx.x;
  const int lane = tid & 31, warp = tid >> 5;
  const unsigned rank = cluster_rank<C>();
  const long long b = static_cast<long long>(blockIdx.x) / C;
  if (b >= L.n_windows) return;  // uniform across the cluster
  if (L.level_idx != nullptr && __ldg(L.level_idx + b) != L.level) return;

  swift_result* out = L.out + b;

  // ---- window sources ----------------------------------------------------
  const TIn* mbase;
  const TIn* rbase;
  if (L.patch_mode) {
    mbase = static_cast<const TIn*>(L.mov) + b * L.mov_stride;
    rbase = static_cast<const TIn*>(L.ref) + b * L.ref_stride;
  } else {
    const int my = __ldg(L.mov_origin + 2 * b), mx = __ldg(L.mov_origin + 2 * b + 1);
    const int ry = __ldg(L.ref_origin + 2 * b), rx = __ldg(L.ref_origin + 2 * b + 1);
    const bool oob = my < 0 || mx < 0 || my > L.mov_h - N || mx > L.mov_w - N || ry < 0 || rx < 0 ||
                     ry > L.ref_h - N || rx > L.ref_w - N;
    if (oob) {
      if (rank == 0 && tid == 0) {
        swift_result r = {0, 0, 0.f, 0.f, 0.f, 0.f, SWIFT_WIN_OUT_OF_BOUNDS, 0};
        *out = r;
      }
      return;
    }
    mbase = static_cast<const TIn*>(L.mov) + static_cast<long long>(my) * L.mov_pitch + mx;
    rbase = static_cast<const TIn*>(L.ref) + static_cast<long long>(ry) * L.ref_pitch + rx;
  }
  const long long mpitch = L.patch_mode ? N : L.mov_pitch;
  const long long rpitch = L.patch_mode ? N : L.ref_pitch;

  // ---- tables -------------------------------------------------------------
  for (int i = tid; i < N; i += T) {
    twid[i] = L.twiddle[i];
    taper[i] = L.taper[i];
  }

  // ---- phase 1: load raw pixels for row pass A, window statistics ---------
  // task (line, j): elements x = j + (N/R1) m of row rank*ROWS + line
  float mraw[P::KA][R1], rraw[P::KA][R1];
  float s_m = 0.f, s_r = 0.f;
  float mn_m = 3.4e38f, mx_m = -3.4e38f, mn_r = 3.4e38f, mx_r = -3.4e38f;
  int bad = 0;
  const float inv_k = 1.0f / static_cast<float>(L.ref_count);
  __syncthreads();  // tables visible
#pragma unroll
  for (int i = 0; i < P::KA; ++i) {
    const int task = tid + i * T;
    const int line = task / (N / R1), j = task % (N / R1);
    const int y = rank * ROWS + line;
    const TIn* mrow = mbase + y * mpitch;
    const TIn* rrow = rbase + y * rpitch;
#pragma unroll
    for (int m = 0; m < R1; ++m) {
      const int x = j + (N / R1) * m;
      mraw[i][m] = load_px<TIn>(mrow + x);
      float rv = load_px<TIn>(rrow + x);
      for (int k = 1; k < L.ref_count; ++k) rv += load_px<TIn>(rrow + k * L.ref_stride + x);
      rraw[i][m] = L.ref_count > 1 ? rv * inv_k : rv;
    }
    const float ay = taper[y];
#pragma unroll
    for (int m = 0; m < R1; ++m) {
      const float a = ay * taper[j + (N / R1) * m];
      s_m = fmaf(a, mraw[i][m], s_m);
      s_r = fmaf(a, rraw[i][m], s_r);
      mn_m = fminf(mn_m, mraw[i][m]);
      mx_m = fmaxf(mx_m, mraw[i][m]);
      mn_r = fminf(mn_r, rraw[i][m]);
      mx_r = fmaxf(mx_r, rraw[i][m]);
      if constexpr (sizeof(TIn) == 4) {
        bad |= !(fabsf(mraw[i][m]) <= 3.4e38f) | !(fabsf(rraw[i][m]) <= 3.4e38f);
      }
    }
  }
  {
    float a = warp_sum_f32(s_m), c = warp_sum_f32(s_r);
    float e = warp_min_f32(mn_m), f = warp_max_f32(mx_m), g = warp_min_f32(mn_r), h = warp_max_f32(mx_r);
    int bb = __any_sync(0xffffffffu, bad);
    if (lane == 0) {
      sc->wsum[warp][0] = a;
      sc->wsum[warp][1] = c;
      sc->wmin[warp][0] = e;
      sc->wmax[warp][0] = f;
      sc->wmin[warp][1] = g;
      sc->wmax[warp][1] = h;
      sc->wbad[warp] = bb;
    }
  }
  __syncthreads();
  if (tid == 0) {
    double a = 0, c = 0;
    float e = 3.4e38f, f = -3.4e38f, g = 3.4e38f, h = -3.4e38f;
    int bb = 0;
    for (int w = 0; w < NW; ++w) {
      a += sc->wsum[w][0];
      c += sc->wsum[w][1];
      e = fminf(e, sc->wmin[w][0]);
      f = fmaxf(f, sc->wmax[w][0]);
      g = fminf(g, sc->wmin[w][1]);
      h = fmaxf(h, sc->wmax[w][1]);
      bb |= sc->wbad[w];
    }
    // all-gather into every CTA of the cluster
    for (unsigned r = 0; r < C; ++r) {
      st_remote_f64<C>(map_rank<C>(smem_addr(&sc->csum[rank][0]), r), a);
      st_remote_f64<C>(map_rank<C>(smem_addr(&sc->csum[rank][1]), r), c);
      st_remote_u64<C>(map_rank<C>(smem_addr(&sc->cmin[rank][0]), r),
                       (static_cast<unsigned long long>(__float_as_uint(g)) << 32) | __float_as_uint(e));
      st_remote_u64<C>(map_rank<C>(smem_addr(&sc->cmax[rank][0]), r),
                       (static_cast<unsigned long long>(__float_as_uint(h)) << 32) | __float_as_uint(f));
      st_remote_u64<C>(map_rank<C>(smem_addr(&sc->ckey[rank]), r), static_cast<unsigned long long>(bb));
    }
  }
  cluster_barrier<C>();
  float mu_m, mu_r;
  {
    double a = 0, c = 0;
    float e = 3.4e38f, f = -3.4e38f, g = 3.4e38f, h = -3.4e38f;
    int bb = 0;
#pragma unroll
    for (int r = 0; r < C; ++r) {
      a += sc->csum[r][0];
      c += sc->csum[r][1];
      e = fminf(e, sc->cmin[r][0]);
      g = fminf(g, sc->cmin[r][1]);
      f = fmaxf(f, sc->cmax[r][0]);
      h = fmaxf(h, sc->cmax[r][1]);
      bb |= static_cast<int>(sc->ckey[r]);
    }
    const int status = bb ? SWIFT_WIN_NONFINITE : ((e == f || g == h) ? SWIFT_WIN_FLAT : SWIFT_WIN_OK);
    if (status != SWIFT_WIN_OK) {
      if (rank == 0 && tid == 0) {
        swift_result r = {0, 0, 0.f, 0.f, 0.f, 0.f, status, 0};
        *out = r;
      }
      cluster_barrier<C>();  // nobody leaves while its slots may still be read
      return;
    }
    mu_m = static_cast<float>(a * L.inv_sum_a);
    mu_r = static_cast<float>(c * L.inv_sum_a);
  }

  // ---- row pass A: apodise, radix-R1 DFT, strided store -------------------
#pragma unroll
  for (int i = 0; i < P::KA; ++i) {
    const int task = tid + i * T;
    const int line = task / (N / R1), j = task % (N / R1);
    const float ay = taper[rank * ROWS + line];
    float2 v[R1];
#pragma unroll
    for (int m = 0; m < R1; ++m) {
      const float a = ay * taper[j + (N / R1) * m];
      v[m] = make_float2(a * (mraw[i][m] - mu_m), a * (rraw[i][m] - mu_r));
    }
    dft<R1, -1>(v);
    float2* row = slab + line * RS;
#pragma unroll
    for (int q = 0; q < R1; ++q) row[P::phys(j * R1 + q)] = v[q];
  }
  __syncthreads();

  // ---- row pass B: twiddle, radix-R2 DFT, hold, push to column owners ----
  {
    float2 h[P::KB][R2];
#pragma unroll
    for (int i = 0; i < P::KB; ++i) {
      const int task = tid + i * T;
      const int line = task / R1, j = task % R1;
      const float2* row = slab + line * RS;
#pragma unroll
      for (int m = 0; m < R2; ++m) {
        float2 x = row[P::phys(j + R1 * m)];
        h[i][m] = m == 0 ? x : cmul(x, twid[m * R1 + j]);
      }
      dft<R2, -1>(h[i]);
    }
    cluster_barrier<C>();  // every CTA finished reading its row slab
    const uint32_t base = smem_addr(slab);
    uint32_t rbase_addr[C];
#pragma unroll
    for (int r = 0; r < C; ++r) rbase_addr[r] = map_rank<C>(base, r);
#pragma unroll
    for (int i = 0; i < P::KB; ++i) {
      const int task = tid + i * T;
      const int line = task / R1, j = task % R1;
      const int y = rank * ROWS + line;
#pragma unroll
      for (int q = 0; q < R2; ++q) {
        const int kx = j + R1 * q;
        int orank, lc;
        P::owner_of(kx, orank, lc);
        uint32_t addr = rbase_addr[0];
#pragma unroll
        for (int r = 1; r < C; ++r) addr = orank == r ? rbase_addr[r] : addr;
        st_remote<C>(addr + static_cast<uint32_t>((y * ROWS + lc) * sizeof(float2)), h[i][q]);
      }
    }
    cluster_barrier<C>();  // column slabs complete
  }

  // ---- column pass A -------------------------------------------------------
  {
    float2 v[P::KA][R1];
#pragma unroll
    for (int i = 0; i < P::KA; ++i) {
      const int task = tid + i * T;
      const int j = task / ROWS, lc = task % ROWS;
#pragma unroll
      for (int m = 0; m < R1; ++m) v[i][m] = slab[(j + (N / R1) * m) * ROWS + lc];
      dft<R1, -1>(v[i]);
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < P::KA; ++i) {
      const int task = tid + i * T;
      const int j = task / ROWS, lc = task % ROWS;
#pragma unroll
      for (int q = 0; q < R1; ++q) slab[(j * R1 + q) * ROWS + lc] = v[i][q];
    }
    __syncthreads();
  }

  // ---- column pass B (in place: each task writes what it read) -------------
#pragma unroll
  for (int i = 0; i < P::KB; ++i) {
    const int task = tid + i * T;
    const int j = task / ROWS, lc = task % ROWS;
    float2 v[R2];
#pragma unroll
    for (int m = 0; m < R2; ++m) {
      float2 x = slab[(j + R1 * m) * ROWS + lc];
      v[m] = m == 0 ? x : cmul(x, twid[m * R1 + j]);
    }
    dft<R2, -1>(v);
#pragma unroll
    for (int q = 0; q < R2; ++q) slab[(j + R1 * q) * ROWS + lc] = v[q];
  }
  __syncthreads();

  // ---- unpack + whiten + inverse column pass A -----------------------------
  // Z = DFT(m' + i r'); with A = Z[k], B = Z[-k]:
  //   C = M conj(R) = ( Im(A B) / 2 , (|A|^2 - |B|^2) / 4 )
  const float half_w = -0.5f * L.w;
  const float inv_n2 = 1.0f / (static_cast<float>(N) * static_cast<float>(N));
  {
    float2 v[P::KAh][R1];
#pragma unroll
    for (int i = 0; i < P::KAh; ++i) {
      const int task = tid + i * T;
      const int j = task / Q, lc = task % Q;
      const bool dc_col = (rank == 0 && lc == 0);
      const int plc = dc_col ? 0 : lc + Q;
#pragma unroll
      for (int m = 0; m < R1; ++m) {
        const int ky = j + (N / R1) * m;
        const int nky = (N - ky) & (N - 1);
        float2 a = slab[ky * ROWS + lc], bb2 = slab[nky * ROWS + plc];
        float2 c = make_float2(0.5f * fmaf(a.x, bb2.y, a.y * bb2.x),
                               0.25f * ((a.x * a.x + a.y * a.y) - (bb2.x * bb2.x + bb2.y * bb2.y)));
        float mag2 = fmaf(c.x, c.x, c.y * c.y);
        float sc1 = mag2 > 0.f ? exp2f(half_w * log2f(mag2)) * inv_n2 : 0.f;
        float2 g = make_float2(c.x * sc1, c.y * sc1);
        if (dc_col) {
          // pack the Nyquist column kx = N/2 as the imaginary part; both are
          // real after the inverse column transform
          float2 a2 = slab[ky * ROWS + Q], b2 = slab[nky * ROWS + Q];
          float2 c2 = make_float2(0.5f * fmaf(a2.x, b2.y, a2.y * b2.x),
                                  0.25f * ((a2.x * a2.x + a2.y * a2.y) - (b2.x * b2.x + b2.y * b2.y)));
          float mq = fmaf(c2.x, c2.x, c2.y * c2.y);
          float sq = mq > 0.f ? exp2f(half_w * log2f(mq)) * inv_n2 : 0.f;
          if (ky == 0) g = make_float2(0.f, 0.f);  // G[0,0] = 0
          g = make_float2(g.x - c2.y * sq, g.y + c2.x * sq);
        }
        v[i][m] = g;
      }
      dft<R1, +1>(v[i]);
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < P::KAh; ++i) {
      const int task = tid + i * T;
      const int j = task / Q, lc = task % Q;
#pragma unroll
      for (int q = 0; q < R1; ++q) slab[(j * R1 + q) * ROWS + lc] = v[i][q];
    }
    __syncthreads();
  }

  // ---- inverse column pass B, hold, push packed row pairs -------------------
  {
    float2 h[P::KBh][R2];
#pragma unroll
    for (int i = 0; i < P::KBh; ++i) {
      const int task = tid + i * T;
      const int j = task / Q, lc = task % Q;
#pragma unroll
      for (int m = 0; m < R2; ++m) {
        float2 x = slab[(j + R1 * m) * ROWS + lc];
        h[i][m] = m == 0 ? x : cmulc(x, twid[m * R1 + j]);
      }
      dft<R2, +1>(h[i]);
    }
    cluster_barrier<C>();  // every CTA finished reading its column slab
    const uint32_t base = smem_addr(slab);
    uint32_t rbase_addr[C];
#pragma unroll
    for (int r = 0; r < C; ++r) rbase_addr[r] = map_rank<C>(base, r);
    constexpr int QP = P::HALF / R1;  // q offset between paired rows
#pragma unroll
    for (int i = 0; i < P::KBh; ++i) {
      const int task = tid + i * T;
      const int j = task / Q, lc = task % Q;
      const int kx = P::kx_of(rank, lc);
      const bool dc_col = (rank == 0 && lc == 0);
#pragma unroll
      for (int q = 0; q < R2; ++q) {
        if ((q % (ROWS / R1)) >= QP) continue;  // q is the first row of a pair
        const int y1 = j + R1 * q;
        const int orank = y1 / ROWS, p = y1 % ROWS;
        uint32_t addr = rbase_addr[0];
#pragma unroll
        for (int r = 1; r < C; ++r) addr = orank == r ? rbase_addr[r] : addr;
        addr += static_cast<uint32_t>(p * RS * sizeof(float2));
        const float2 h1 = h[i][q], h2 = h[i][q + QP];
        if (dc_col) {
          st_remote<C>(addr + P::phys(0) * sizeof(float2), make_float2(h1.x, h2.x));
          st_remote<C>(addr + P::phys(N / 2) * sizeof(float2), make_float2(h1.y, h2.y));
        } else {
          st_remote<C>(addr + P::phys(kx) * sizeof(float2), make_float2(h1.x - h2.y, h1.y + h2.x));
          st_remote<C>(addr + P::phys(N - kx) * sizeof(float2), make_float2(h1.x + h2.y, h2.x - h1.y));
        }
      }
    }
    cluster_barrier<C>();  // packed rows complete
  }

  // ---- inverse row pass A on packed rows -----------------------------------
  {
    float2 v[P::KAh][R1];
#pragma unroll
    for (int i = 0; i < P::KAh; ++i) {
      const int task = tid + i * T;
      const int line = task / (N / R1), j = task % (N / R1);
      const float2* row = slab + line * RS;
#pragma unroll
      for (int m = 0; m < R1; ++m) v[i][m] = row[P::phys(j + (N / R1) * m)];
      dft<R1, +1>(v[i]);
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < P::KAh; ++i) {
      const int task = tid + i * T;
      const int line = task / (N / R1), j = task % (N / R1);
      float2* row = slab + line * RS;
#pragma unroll
      for (int q = 0; q < R1; ++q) row[P::phys(j * R1 + q)] = v[i][q];
    }
    __syncthreads();
  }

  // ---- inverse row pass B -> surface, argmax --------------------------------
  float* surf = reinterpret_cast<float*>(slab + P::PACKED);  // [ROWS][N]
  float sv[P::KBh][2][R2];
  unsigned long long best = 0ull;
#pragma unroll
  for (int i = 0; i < P::KBh; ++i) {
    const int task = tid + i * T;
    const int line = task / R1, j = task % R1;
    const float2* row = slab + line * RS;
    float2 v[R2];
#pragma unroll
    for (int m = 0; m < R2; ++m) {
      float2 x = row[P::phys(j + R1 * m)];
      v[m] = m == 0 ? x : cmulc(x, twid[m * R1 + j]);
    }
    dft<R2, +1>(v);
    const int l1 = line, l2 = line + P::HALF;
    const int y1 = rank * ROWS + l1, y2 = rank * ROWS + l2;
#pragma unroll
    for (int q = 0; q < R2; ++q) {
      const int x = j + R1 * q;
      sv[i][0][q] = v[q].x;
      sv[i][1][q] = v[q].y;
      surf[l1 * N + x] = v[q].x;
      surf[l2 * N + x] = v[q].y;
      unsigned long long k1 = argmax_key(v[q].x, static_cast<uint32_t>(y1 * N + x));
      unsigned long long k2 = argmax_key(v[q].y, static_cast<uint32_t>(y2 * N + x));
      best = k1 > best ? k1 : best;
      best = k2 > best ? k2 : best;
    }
  }
  best = warp_max_u64(best);
  if (lane == 0) sc->wkey[warp] = best;
  __syncthreads();
  if (tid == 0) {
    unsigned long long bk = 0ull;
    for (int w = 0; w < NW; ++w) bk = sc->wkey[w] > bk ? sc->wkey[w] : bk;
    for (unsigned r = 0; r < C; ++r) st_remote_u64<C>(map_rank<C>(smem_addr(&sc->ckey[rank]), r), bk);
  }
  cluster_barrier<C>();
  unsigned long long gk = 0ull;
#pragma unroll
  for (int r = 0; r < C; ++r) gk = sc->ckey[r] > gk ? sc->ckey[r] : gk;
  const uint32_t pidx = key_index(gk);
  const int py = static_cast<int>(pidx / N), px = static_cast<int>(pidx % N);

  // ---- SNR background partials (outside the exclusion disc) ---------------
  {
    float s1 = 0.f, s2 = 0.f, cnt = 0.f;
#pragma unroll
    for (int i = 0; i < P::KBh; ++i) {
      const int task = tid + i * T;
      const int line = task / R1, j = task % R1;
#pragma unroll
      for (int h2 = 0; h2 < 2; ++h2) {
        const int y = rank * ROWS + line + h2 * P::HALF;
        int dy = abs(y - py);
        dy = min(dy, N - dy);
#pragma unroll
        for (int q = 0; q < R2; ++q) {
          const int x = j + R1 * q;
          int dx = abs(x - px);
          dx = min(dx, N - dx);
          const float d2 = static_cast<float>(dy * dy + dx * dx);
          const float s = sv[i][h2][q];
          if (d2 > L.radius2) {
            s1 += s;
            s2 = fmaf(s, s, s2);
            cnt += 1.f;
          }
        }
      }
    }
    double a = warp_sum_f64(static_cast<double>(s1));
    double c = warp_sum_f64(static_cast<double>(s2));
    double n = warp_sum_f64(static_cast<double>(cnt));
    if (lane == 0) {
      sc->wbg[warp][0] = a;
      sc->wbg[warp][1] = c;
      sc->wbg[warp][2] = n;
    }
  }
  __syncthreads();
  if (tid == 0) {
    double a = 0, c = 0, n = 0;
    for (int w = 0; w < NW; ++w) {
      a += sc->wbg[w][0];
      c += sc->wbg[w][1];
      n += sc->wbg[w][2];
    }
    const uint32_t dst = map_rank<C>(smem_addr(&sc->cbg[rank][0]), 0);
    st_remote_f64<C>(dst, a);
    st_remote_f64<C>(dst + 8, c);
    st_remote_f64<C>(dst + 16, n);
    // peak neighbours owned by this CTA go to rank 0
    const int ys[4] = {(py + N - 1) & (N - 1), (py + 1) & (N - 1), py, py};
    const int xs[4] = {px, px, (px + N - 1) & (N - 1), (px + 1) & (N - 1)};
    for (int k = 0; k < 4; ++k) {
      if (ys[k] / ROWS == static_cast<int>(rank)) {
        const float v = surf[(ys[k] % ROWS) * N + xs[k]];
        const uint32_t d = map_rank<C>(smem_addr(&sc->nb[k]), 0);
        if constexpr (C == 1) {
          sc->nb[k] = v;
        } else {
          asm volatile("st.shared::cluster.f32 [%0], %1;" ::"r"(d), "f"(v) : "memory");
        }
      }
    }
  }
  cluster_barrier<C>();
  if (rank == 0 && tid == 0) {
    double a = 0, c = 0, n = 0;
    for (int r = 0; r < C; ++r) {
      a += sc->cbg[r][0];
      c += sc->cbg[r][1];
      n += sc->cbg[r][2];
    }
    const double mu = a / n;
    double var = c / n - mu * mu;
    const double pk = static_cast<double>(key_value(gk));
    double snr;
    if (var > 0.0) {
      snr = (pk - mu) / sqrt(var);
    } else {
      snr = pk > mu ? __longlong_as_double(0x7ff0000000000000ll) : 0.0;
    }
    auto parab = [](double sm, double s0, double sp) -> double {
      const double den = sm - 2.0 * s0 + sp;
      if (!(den < 0.0)) return 0.0;
      double d = 0.5 * (sm - sp) / den;
      return d < -0.5 ? -0.5 : (d > 0.5 ? 0.5 : d);
    };
    const double fy = parab(sc->nb[0], pk, sc->nb[1]);
    const double fx = parab(sc->nb[2], pk, sc->nb[3]);
    const int dy = py < N / 2 ? py : py - N;
    const int dx = px < N / 2 ? px : px - N;
    swift_result r;
    r.dy = dy;
    r.dx = dx;
    r.sy = static_cast<float>(dy + fy);
    r.sx = static_cast<float>(dx + fx);
    r.snr = static_cast<float>(snr);
    r.peak = static_cast<float>(pk);
    r.status = SWIFT_WIN_OK;
    r.reserved = 0;
    *out = r;
  }
}

}  // namespace swift
