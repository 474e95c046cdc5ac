// Launchers of the streaming forward path (five kernels per slice of windows).
#include "swim_stream.cuh"

namespace swift {

namespace {

size_t align256(size_t x) { return (x + 255) & ~static_cast<size_t>(255); }

// cuTensorMapEncodeTiled from the driver, fetched once through the runtime
// (the library links no driver library); null when the driver has none
using EncodeTiled = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                 const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiled encode_tiled() {
  static const EncodeTiled fn = [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess) {
      cudaGetLastError();
      p = nullptr;
    }
    return reinterpret_cast<EncodeTiled>(p);
  }();
  return fn;
}

// The tile map of one uint8 section image (RowMaps): [h][w / 16][16] bytes,
// box [rb][n / 16 + 1][16]; false where the image's address, pitch or width
// is not a multiple of 16 bytes or the driver refuses the map.
bool tile_map(CUtensorMap* m, const void* data, int h, int w, long long pitch, int n, int rb) {
  const EncodeTiled enc = encode_tiled();
  if (!enc || !data || h < 1 || w < 16 || (reinterpret_cast<uintptr_t>(data) & 15) || (pitch & 15) || (w & 15) ||
      pitch < w)
    return false;
  const cuuint64_t dim[3] = {16, static_cast<cuuint64_t>(w / 16), static_cast<cuuint64_t>(h)};
  const cuuint64_t stride[2] = {16, static_cast<cuuint64_t>(pitch)};
  const cuuint32_t box[3] = {16, static_cast<cuuint32_t>(n / 16 + 1), static_cast<cuuint32_t>(rb)};
  const cuuint32_t estride[3] = {1, 1, 1};
  return enc(m, CU_TENSOR_MAP_DATA_TYPE_UINT8, 3, const_cast<void*>(data), dim, stride, box, estride,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// The row kernel's tensor maps for a launch: uint8 section windows with a
// one-section reference, when MatchLaunch::row_tma asks for them
template <int N, typename TIn>
RowMaps row_maps(const MatchLaunch& L) {
  RowMaps M{};
  if constexpr (sizeof(TIn) == 1) {
    if (L.row_tma == 0 || L.patch_mode || L.ref_count != 1) return M;
    constexpr int RB = StreamGeom<N>::RB;
    if (!tile_map(&M.mov, L.mov, L.mov_h, L.mov_w, L.mov_pitch, N, RB) ||
        !tile_map(&M.ref, L.ref, L.ref_h, L.ref_w, L.ref_pitch, N, RB))
      return RowMaps{};
    M.on = 1;
    M.all = L.row_tma == 2 ? 1 : 0;
  }
  return M;
}

template <int N>
size_t part_blocks() {
  return StreamGeom<N>::NB3;
}

size_t blocks3(int n) {
  switch (n) {
    case 64:
      return StreamGeom<64>::NB3;
    case 128:
      return StreamGeom<128>::NB3;
    case 512:
      return StreamGeom<512>::NB3;
    default:
      return StreamGeom<256>::NB3;
  }
}

template <int N, typename TIn>
cudaError_t launch_n(const MatchLaunch& L, const StreamWork& W, cudaStream_t st) {
  using G = StreamGeom<N>;
  const unsigned S = static_cast<unsigned>(W.count);
  if (S == 0) return cudaSuccess;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  // n <= 256: column pairs unpacked at load (whitening and the first inverse
  // pass in registers); n = 512 keeps the per-column kernel (its pass B would
  // hold 2 x 32 complex values per thread)
  constexpr bool kPair = N <= 256;
  // n <= 256, plain forward: no statistics kernel (the row kernel records
  // each block's sums and flatness, the column-pair kernel combines them and
  // removes the means in the spectrum)
  const bool fold_stats = kPair && stream_stats_folded(N, L) && W.rstat != nullptr;
  static unsigned m1 = 0, m2 = 0, m3 = 0, m4 = 0, m5 = 0, m6 = 0;
  if ((e = smem_optin(stream_rows_kernel<N, TIn>, rows_smem<N, TIn>(), m1, dev)) != cudaSuccess) return e;
  if constexpr (kPair) {
    if ((e = smem_optin(stream_rows_kernel<N, TIn, true>, rows_smem<N, TIn>(), m5, dev)) != cudaSuccess) return e;
    if ((e = smem_optin(stream_cpair_kernel<N>, cpair_smem<N>(), m2, dev)) != cudaSuccess) return e;
    if ((e = smem_optin(stream_cpair_kernel<N, true>, cpair_smem<N>(), m6, dev)) != cudaSuccess) return e;
  } else {
    if ((e = smem_optin(stream_cols_kernel<N>, cols_smem<N>(), m2, dev)) != cudaSuccess) return e;
  }
  if ((e = smem_optin(stream_irows_kernel<N, false>, irows_smem<N>(), m3, dev)) != cudaSuccess) return e;
  if ((e = smem_optin(stream_peak_kernel<N>, peak_smem<N>(), m4, dev)) != cudaSuccess) return e;
  auto mark = [&](int k) {
    if (W.ev) cudaEventRecord(W.ev[k], st);
  };
  const RowMaps M = row_maps<N, TIn>(L);
  mark(0);
  if (!fold_stats) stream_stats_kernel<N, TIn><<<S, 256, 0, st>>>(L, W);
  mark(1);
  if constexpr (kPair) {
    if (fold_stats) {
      stream_rows_kernel<N, TIn, true><<<S * (N / G::RB), 256, rows_smem<N, TIn>(), st>>>(L, W, M);
    } else {
      stream_rows_kernel<N, TIn><<<S * (N / G::RB), 256, rows_smem<N, TIn>(), st>>>(L, W, M);
    }
  } else {
    stream_rows_kernel<N, TIn><<<S * (N / G::RB), 256, rows_smem<N, TIn>(), st>>>(L, W, M);
  }
  mark(2);
  if constexpr (kPair) {
    if (fold_stats) {
      stream_cpair_kernel<N, true><<<S * PairGeom<N>::NB, PairGeom<N>::T, cpair_smem<N>(), st>>>(L, W);
    } else {
      stream_cpair_kernel<N><<<S * PairGeom<N>::NB, PairGeom<N>::T, cpair_smem<N>(), st>>>(L, W);
    }
  } else {
    stream_cols_kernel<N><<<S * G::NB2, G::T2, cols_smem<N>(), st>>>(L, W);
  }
  mark(3);
  {
    StreamWork W3 = W;
    if (!(N <= 256 && L.radius2 < 64.f)) W3.done = nullptr;
    stream_irows_kernel<N, false><<<S * G::NB3, 256, irows_smem<N>(), st>>>(L, W3);
  }
  mark(4);
  // n <= 256, exclusion radius below 8 px, block counters given: the last
  // inverse-row block of each window finalizes it; otherwise a kernel of its own
  const bool fold = N <= 256 && W.done != nullptr && L.radius2 < 64.f;
  if (!fold) stream_peak_kernel<N><<<S, PeakGeom<N>::T, peak_smem<N>(), st>>>(L, W);
  mark(5);
  return cudaGetLastError();
}

}  // namespace

// row blocks of a window (the row kernel's CTAs per window)
size_t row_blocks(int n) {
  switch (n) {
    case 64:
      return 64 / StreamGeom<64>::RB;
    case 128:
      return 128 / StreamGeom<128>::RB;
    case 512:
      return 512 / StreamGeom<512>::RB;
    default:
      return 256 / StreamGeom<256>::RB;
  }
}

size_t stream_bytes_per_window(int n) {
  const size_t nn = static_cast<size_t>(n) * n;
  return sizeof(float4) + sizeof(float2) * nn + sizeof(float2) * nn / 2 + 3 * sizeof(unsigned long long) * blocks3(n) +
         8 * sizeof(float) * row_blocks(n);
}

StreamWork stream_carve(void* base, long long capacity, int n, long long b0, long long count) {
  const size_t nn = static_cast<size_t>(n) * n;
  unsigned char* p = static_cast<unsigned char*>(base);
  StreamWork W;
  W.stats = reinterpret_cast<float4*>(p);
  p += align256(sizeof(float4) * capacity);
  W.zr = reinterpret_cast<float2*>(p);
  p += align256(sizeof(float2) * nn * capacity);
  W.h = reinterpret_cast<float2*>(p);
  p += align256(sizeof(float2) * nn / 2 * capacity);
  W.part = reinterpret_cast<unsigned long long*>(p);
  p += align256(3 * sizeof(unsigned long long) * blocks3(n) * capacity);
  W.rstat = reinterpret_cast<float*>(p);
  W.b0 = b0;
  W.count = count;
  return W;
}

bool stream_radices(int n, int* r1, int* r2) {
  switch (n) {
    case 64:
      *r1 = StreamGeom<64>::R1, *r2 = StreamGeom<64>::R2;
      return true;
    case 128:
      *r1 = StreamGeom<128>::R1, *r2 = StreamGeom<128>::R2;
      return true;
    case 256:
      *r1 = StreamGeom<256>::R1, *r2 = StreamGeom<256>::R2;
      return true;
    case 512:
      *r1 = StreamGeom<512>::R1, *r2 = StreamGeom<512>::R2;
      return true;
    default:
      return false;
  }
}

namespace {
__global__ void __launch_bounds__(256) taper_spectrum_kernel(int n, int apod, float alpha, const float* taper,
                                                             float* out) {
  __shared__ float cos_tab[512];
  __shared__ float tap[512];
  for (int j = threadIdx.x; j < n; j += blockDim.x) tap[j] = taper[j];
  __syncthreads();
  taper_spectrum(n, apod, alpha, tap, out, cos_tab, threadIdx.x, blockDim.x);
}
}  // namespace

cudaError_t launch_taper_spectrum(int n, int apod, float alpha, const float* taper, float* out, cudaStream_t stream) {
  if (n < 2 || n > 512 || (n & (n - 1)) != 0) return cudaErrorInvalidValue;
  taper_spectrum_kernel<<<1, 256, 0, stream>>>(n, apod, alpha, taper, out);
  return cudaGetLastError();
}

cudaError_t launch_stream(int n, swift_dtype dtype, const MatchLaunch& L, const StreamWork& W, cudaStream_t st) {
  const bool u8 = dtype == SWIFT_IN_U8;
  switch (n) {
    case 64:
      return u8 ? launch_n<64, uint8_t>(L, W, st) : launch_n<64, float>(L, W, st);
    case 128:
      return u8 ? launch_n<128, uint8_t>(L, W, st) : launch_n<128, float>(L, W, st);
    case 256:
      return u8 ? launch_n<256, uint8_t>(L, W, st) : launch_n<256, float>(L, W, st);
    case 512:
      return u8 ? launch_n<512, uint8_t>(L, W, st) : launch_n<512, float>(L, W, st);
    default:
      return cudaErrorInvalidValue;
  }
}

}  // namespace swift
