// Launch helpers shared by the kernel translation units.
#pragma once
#include <cuda_runtime.h>

#include "gbd_tc.cuh"
#include "gbd_kernels.cuh"

namespace gbd {

__host__ __device__ constexpr int min_blocks(int T) { return T >= 768 ? 1 : 768 / T; }
// The FP32 convolution kernels run at 1152 threads per SM (three blocks of 384 at <= 56
// registers): the film's fused pass holds at most two components' values at a time, and the
// 3D z convolution splits its fused pass into per-component butterflies and a product phase.
__host__ __device__ constexpr int min_blocks_film(int T) { return T >= 1152 ? 1 : 1152 / T; }

// Raises the dynamic shared-memory limit of kernel k once per (kernel, device). Meshes call
// this for their kernels when they are created, so launches inside a stream capture find the
// attribute already set.
bool prep_seen(const void* k, int dev);
template <class K>
static void prep(K k, size_t smem) {
  int dev = 0;
  cudaGetDevice(&dev);
  if (prep_seen((const void*)k, dev)) return;
  cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

}  // namespace gbd
