// Instantiations and launchers of the fused forward matching kernel.
#include "swim_kernel.cuh"

namespace swift {

namespace {

// Persistent grid: as many clusters (or CTAs) as can be resident at once.
template <int N, int C, typename TIn, bool BULK>
cudaError_t resident_clusters(int device, int* out) {
  static int cached[32] = {};
  if (device < 32 && cached[device] > 0) {
    *out = cached[device];
    return cudaSuccess;
  }
  auto kern = swim_forward_kernel<N, C, TIn, BULK>;
  constexpr size_t smem = forward_smem_bytes<N, C, BULK>();
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
  if (e != cudaSuccess) return e;
  int n = 0;
  if (C > 1) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(C, 1, 1);
    cfg.blockDim = dim3(Plan2D<N, C>::T, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    e = cudaOccupancyMaxActiveClusters(&n, kern, &cfg);
    if (e != cudaSuccess) return e;
  } else {
    int per_sm = 0, sms = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, Plan2D<N, C>::T, smem);
    if (e != cudaSuccess) return e;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    if (e != cudaSuccess) return e;
    n = per_sm * sms;
  }
  if (n < 1) return cudaErrorInvalidConfiguration;
  if (device < 32) cached[device] = n;
  *out = n;
  return cudaSuccess;
}

template <int N, int C, typename TIn, bool BULK>
cudaError_t launch_one(const MatchLaunch& L, cudaStream_t stream) {
  if (L.n_windows <= 0) return cudaSuccess;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  int clusters = 0;
  e = resident_clusters<N, C, TIn, BULK>(dev, &clusters);
  if (e != cudaSuccess) return e;
  const long long g = L.n_windows < clusters ? L.n_windows : clusters;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(static_cast<unsigned>(g * C), 1, 1);
  cfg.blockDim = dim3(Plan2D<N, C>::T, 1, 1);
  cfg.dynamicSmemBytes = forward_smem_bytes<N, C, BULK>();
  cfg.stream = stream;
  cudaLaunchAttribute attr[1];
  if (C > 1) {
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
  }
  return cudaLaunchKernelEx(&cfg, swim_forward_kernel<N, C, TIn, BULK>, L);
}

template <int N, int C>
cudaError_t launch_size(swift_dtype dtype, bool bulk, const MatchLaunch& L, cudaStream_t stream) {
  if (dtype == SWIFT_IN_F32) return launch_one<N, C, float, false>(L, stream);
  return bulk ? launch_one<N, C, uint8_t, true>(L, stream) : launch_one<N, C, uint8_t, false>(L, stream);
}

}  // namespace

cudaError_t launch_forward(int n, swift_dtype dtype, bool bulk, const MatchLaunch& L, cudaStream_t stream) {
  switch (n) {
    case 64:
      return launch_size<64, 1>(dtype, bulk, L, stream);
    case 128:
      return launch_size<128, 2>(dtype, bulk, L, stream);
    case 256:
      return launch_size<256, 8>(dtype, bulk, L, stream);
    default:
      return cudaErrorInvalidValue;
  }
}

bool forward_radices(int n, int* r1, int* r2) {
  switch (n) {
    case 64:
      *r1 = Geometry<64, 1>::R1;
      *r2 = Geometry<64, 1>::R2;
      return true;
    case 128:
      *r1 = Geometry<128, 2>::R1;
      *r2 = Geometry<128, 2>::R2;
      return true;
    case 256:
      *r1 = Geometry<256, 8>::R1;
      *r2 = Geometry<256, 8>::R2;
      return true;
    default:
      return false;
  }
}

}  // namespace swift
