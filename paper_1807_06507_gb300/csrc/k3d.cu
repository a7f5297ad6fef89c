// k3d.cu -- instantiations and launch of the fused 3-D correlation kernel.
#include "k3d.cuh"
#include "devonce.h"
#include "launch.h"

namespace swc {

template <int K>
static cudaError_t launch_k(const K3DParams& p, int grid, size_t smem, cudaStream_t st) {
  static std::atomic<uint64_t> attr_done{0};  // one bit per device
  cudaError_t e = once_per_device(attr_done, [] {
    return cudaFuncSetAttribute(k3d_kernel<kTY3, tx3<K>(), K, K, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  });
  if (e != cudaSuccess) return e;
  k3d_kernel<kTY3, tx3<K>(), K, K, false><<<grid, K3_THREADS, smem, st>>>(p);
  return cudaGetLastError();
}

template <int K>
static void geo(Geo3DInfo* g) {
  using G = Geo3D<kTY3, tx3<K>(), K, K>;
  g->TY = kTY3;
  g->TX = tx3<K>();
  g->TYI = G::TYI;
  g->BXW = G::BXW;
  g->XH = G::XH;
  g->VSP = G::VSP;
}

#define SWC_K3D_CASES(X) X(1) X(3) X(5) X(7) X(9) X(11) X(13) X(15)

bool k3d_geometry(int k, Geo3DInfo* g) {
  switch (k) {
#define X(K) \
  case K:    \
    geo<K>(g); \
    return true;
    SWC_K3D_CASES(X)
#undef X
    default:
      return false;
  }
}

cudaError_t k3d_launch(int k, const K3DParams& p, int grid, size_t smem, cudaStream_t st) {
  switch (k) {
#define X(K) \
  case K:    \
    return launch_k<K>(p, grid, smem, st);
    SWC_K3D_CASES(X)
#undef X
    default:
      return cudaErrorInvalidValue;
  }
}

int k3d_blocks_per_sm(int k, size_t smem) {
  int b = 0;
  cudaError_t e = cudaErrorInvalidValue;
  switch (k) {
#define X(K)                                                                                        \
  case K:                                                                                           \
    e = cudaFuncSetAttribute(k3d_kernel<kTY3, tx3<K>(), K, K, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                             200 * 1024);                                                           \
    if (e == cudaSuccess)                                                                           \
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k3d_kernel<kTY3, tx3<K>(), K, K, false>, K3_THREADS, smem); \
    break;
    SWC_K3D_CASES(X)
#undef X
    default:
      break;
  }
  return e == cudaSuccess ? b : 0;
}

}  // namespace swc
