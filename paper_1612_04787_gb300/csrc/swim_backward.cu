// Launchers of the affine-warp preparation, the forward on prepared windows,
// and the backward pass.
#include "swim_backward.cuh"

namespace swift {

namespace {

size_t align256(size_t x) { return (x + 255) & ~static_cast<size_t>(255); }

int nb3(int n) {
  return n == 64 ? StreamGeom<64>::NB3 : (n == 128 ? StreamGeom<128>::NB3 : StreamGeom<256>::NB3);
}
int nb6(int n) {
  return n == 64 ? BackColGeom<64>::NB : (n == 128 ? BackColGeom<128>::NB : BackColGeom<256>::NB);
}

template <int N>
constexpr size_t grows_smem() {
  return sizeof(float2) * (StreamGeom<N>::PB * StreamGeom<N>::RS + N);
}
template <int N>
constexpr size_t gcols_smem() {
  return sizeof(float2) * (N * BackColGeom<N>::LS + 2 * N);
}
template <int N>
constexpr size_t ginv_smem() {
  return sizeof(float2) * (StreamGeom<N>::PB * StreamGeom<N>::RS + N) + sizeof(float) * N;
}

// the streaming launch description for the prepared float32 windows of a slice
MatchLaunch prepared(const MatchLaunch& L, const BackWork& BW, int n, long long b0) {
  MatchLaunch P = L;
  P.ref = BW.rp;
  P.mov = BW.mp;
  P.ref_pitch = P.mov_pitch = n;
  P.ref_stride = P.mov_stride = static_cast<long long>(n) * n;
  P.ref_count = 1;
  P.patch_mode = 1;
  P.level_idx = L.level_idx ? L.level_idx + b0 : nullptr;
  P.out = L.out ? L.out + b0 : nullptr;
  P.pre_status = BW.pre_status;
  return P;
}

template <int N, typename TIn>
cudaError_t prepare_n(const MatchLaunch& L, const BackLaunch& K, const BackWork& BW, long long b0, cudaStream_t st) {
  const unsigned S = static_cast<unsigned>(BW.fw.count);
  if (S == 0) return cudaSuccess;
  prep_kernel<N, TIn><<<S * (N / 16), 256, 0, st>>>(L, K, BW, b0);
  return cudaGetLastError();
}

template <int N, typename TIn>
cudaError_t backward_n(const MatchLaunch& L, const BackLaunch& K, const BackWork& BW, long long b0,
                       cudaStream_t st) {
  using G = StreamGeom<N>;
  const unsigned S = static_cast<unsigned>(BW.fw.count);
  if (S == 0) return cudaSuccess;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  static unsigned m1 = 0, m2 = 0, m3 = 0, m4 = 0, m5 = 0, m6 = 0;
  if ((e = smem_optin(stream_rows_kernel<N, float>, rows_smem<N, float>(), m1, dev)) != cudaSuccess) return e;
  if ((e = smem_optin(stream_cols_kernel<N, true>, cols_smem<N>(), m2, dev)) != cudaSuccess) return e;
  if ((e = smem_optin(stream_irows_kernel<N>, irows_smem<N>(), m3, dev)) != cudaSuccess) return e;
  if ((e = smem_optin(back_grows_kernel<N>, grows_smem<N>(), m4, dev)) != cudaSuccess) return e;
  if ((e = smem_optin(back_gcols_kernel<N>, gcols_smem<N>(), m5, dev)) != cudaSuccess) return e;
  if ((e = smem_optin(back_grows_inv_kernel<N>, ginv_smem<N>(), m6, dev)) != cudaSuccess) return e;
  const MatchLaunch P = prepared(L, BW, N, b0);
  StreamWork W = BW.fw;
  W.b0 = 0;
  // forward recompute, keeping C and R
  stream_stats_kernel<N, float><<<S, 256, 0, st>>>(P, W);
  stream_rows_kernel<N, float><<<S * (N / G::RB), 256, rows_smem<N, float>(), st>>>(P, W, RowMaps{});
  stream_cols_kernel<N, true><<<S * G::NB2, G::T2, cols_smem<N>(), st>>>(P, W, BW.cr);
  stream_irows_kernel<N><<<S * G::NB3, 256, irows_smem<N>(), st>>>(P, W);
  back_stats_kernel<N><<<S, 32, 0, st>>>(P, W, BW.bst);
  // adjoint
  back_grows_kernel<N><<<S * G::NB3, 256, grows_smem<N>(), st>>>(P, K, BW, b0);
  back_gcols_kernel<N><<<S * BackColGeom<N>::NB, 256, gcols_smem<N>(), st>>>(P, BW);
  back_grows_inv_kernel<N><<<S * G::NB3, 256, ginv_smem<N>(), st>>>(P, BW);
  back_affine_kernel<N, TIn><<<S, 256, 0, st>>>(L, K, BW, b0);
  back_wsum_kernel<<<1, 256, 0, st>>>(BW, S, K.gw_acc);
  return cudaGetLastError();
}

}  // namespace

size_t back_bytes_per_window(int n) {
  const size_t nn = static_cast<size_t>(n) * n;
  const size_t w2 = static_cast<size_t>(n) * (n / 2 + 1);
  return stream_bytes_per_window(n) + 2 * sizeof(float) * nn + sizeof(int) + 2 * sizeof(float2) * w2 +
         8 * sizeof(double) + sizeof(float2) * w2 + sizeof(double) * (nb6(n) + nb3(n) + 1);
}

BackWork back_carve(void* base, long long capacity, int n, long long count) {
  const size_t nn = static_cast<size_t>(n) * n;
  const size_t w2 = static_cast<size_t>(n) * (n / 2 + 1);
  unsigned char* p = static_cast<unsigned char*>(base);
  BackWork BW;
  BW.fw = stream_carve(p, capacity, n, 0, count);
  p += align256(stream_bytes_per_window(n) * capacity + 4 * 256);
  BW.mp = reinterpret_cast<float*>(p);
  p += align256(sizeof(float) * nn * capacity);
  BW.rp = reinterpret_cast<float*>(p);
  p += align256(sizeof(float) * nn * capacity);
  BW.pre_status = reinterpret_cast<int*>(p);
  p += align256(sizeof(int) * capacity);
  BW.cr = reinterpret_cast<float2*>(p);
  p += align256(2 * sizeof(float2) * w2 * capacity);
  BW.bst = reinterpret_cast<double*>(p);
  p += align256(8 * sizeof(double) * capacity);
  BW.gr = reinterpret_cast<float2*>(p);
  p += align256(sizeof(float2) * w2 * capacity);
  BW.gwp = reinterpret_cast<double*>(p);
  p += align256(sizeof(double) * nb6(n) * capacity);
  BW.gsum = reinterpret_cast<double*>(p);
  p += align256(sizeof(double) * nb3(n) * capacity);
  BW.gwin = reinterpret_cast<double*>(p);
  return BW;
}

cudaError_t launch_prepare(int n, swift_dtype dtype, const MatchLaunch& L, const BackLaunch& K, const BackWork& BW,
                           long long b0, cudaStream_t st) {
  const bool u8 = dtype == SWIFT_IN_U8;
  switch (n) {
    case 64:
      return u8 ? prepare_n<64, uint8_t>(L, K, BW, b0, st) : prepare_n<64, float>(L, K, BW, b0, st);
    case 128:
      return u8 ? prepare_n<128, uint8_t>(L, K, BW, b0, st) : prepare_n<128, float>(L, K, BW, b0, st);
    case 256:
      return u8 ? prepare_n<256, uint8_t>(L, K, BW, b0, st) : prepare_n<256, float>(L, K, BW, b0, st);
    default:
      return cudaErrorInvalidValue;
  }
}

cudaError_t launch_prepared_forward(int n, const MatchLaunch& L, const BackWork& BW, long long b0,
                                    cudaStream_t st) {
  const MatchLaunch P = prepared(L, BW, n, b0);
  StreamWork W = BW.fw;
  W.b0 = 0;
  return launch_stream(n, SWIFT_IN_F32, P, W, st);
}

cudaError_t launch_backward(int n, swift_dtype dtype, const MatchLaunch& L, const BackLaunch& K, const BackWork& BW,
                            long long b0, cudaStream_t st) {
  const bool u8 = dtype == SWIFT_IN_U8;
  switch (n) {
    case 64:
      return u8 ? backward_n<64, uint8_t>(L, K, BW, b0, st) : backward_n<64, float>(L, K, BW, b0, st);
    case 128:
      return u8 ? backward_n<128, uint8_t>(L, K, BW, b0, st) : backward_n<128, float>(L, K, BW, b0, st);
    case 256:
      return u8 ? backward_n<256, uint8_t>(L, K, BW, b0, st) : backward_n<256, float>(L, K, BW, b0, st);
    default:
      return cudaErrorInvalidValue;
  }
}

namespace {
__global__ void wout_kernel(const double* acc, float* out, int n) {
  const int i = threadIdx.x;
  if (i < n) out[i] = static_cast<float>(acc[i]);
}
}  // namespace

cudaError_t launch_wout(const double* acc, float* out, int n, cudaStream_t st) {
  wout_kernel<<<1, 32, 0, st>>>(acc, out, n);
  return cudaGetLastError();
}

}  // namespace swift
