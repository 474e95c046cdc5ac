// Instantiations and launchers of the fused forward matching kernel.
#include "swim_kernel.cuh"

namespace swift {

template <int N, int C>
static constexpr size_t forward_smem_bytes() {
  using P = Plan2D<N, C>;
  return sizeof(float2) * (P::SLAB + N) + sizeof(float) * N + sizeof(Scratch);
}

template <int N, int C, typename TIn>
static cudaError_t launch_one(const MatchLaunch& L, cudaStream_t stream) {
  auto kern = swim_forward_kernel<N, C, TIn>;
  constexpr size_t smem = forward_smem_bytes<N, C>();
  // the shared-memory opt-in is a per-device function attribute: set it once per device
  static unsigned attr_done = 0u;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev >= 32 || !(attr_done & (1u << dev))) {
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    if (dev < 32) attr_done |= 1u << dev;
  }
  if (L.n_windows <= 0) return cudaSuccess;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(static_cast<unsigned>(L.n_windows * C), 1, 1);
  cfg.blockDim = dim3(Plan2D<N, C>::T, 1, 1);
  cfg.dynamicSmemBytes = smem;
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
  return cudaLaunchKernelEx(&cfg, kern, L);
}

cudaError_t launch_forward(int n, swift_dtype dtype, const MatchLaunch& L, cudaStream_t stream) {
  const bool u8 = dtype == SWIFT_IN_U8;
  switch (n) {
    case 64:
      return u8 ? launch_one<64, 1, uint8_t>(L, stream) : launch_one<64, 1, float>(L, stream);
    case 128:
      return u8 ? launch_one<128, 1, uint8_t>(L, stream) : launch_one<128, 1, float>(L, stream);
    case 256:
      return u8 ? launch_one<256, 4, uint8_t>(L, stream) : launch_one<256, 4, float>(L, stream);
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
      *r1 = Geometry<128, 1>::R1;
      *r2 = Geometry<128, 1>::R2;
      return true;
    case 256:
      *r1 = Geometry<256, 4>::R1;
      *r2 = Geometry<256, 4>::R2;
      return true;
    default:
      return false;
  }
}

}  // namespace swift
