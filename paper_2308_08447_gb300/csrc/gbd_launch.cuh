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

// Programmatic dependent launch (PTX griddepcontrol): the x-row kernels, the film convolution and
// the extrapolated RK stage are launched with programmatic stream serialization, so a launch may
// begin while the kernel before it in the stream still runs -- its blocks become resident on SMs
// the predecessor has left idle. Every thread waits for the predecessor grid to complete with its
// memory operations visible before it touches memory the predecessor may write; the block then
// allows its own successor to launch. Since no block releases its successor before its own wait
// returns, a kernel that has started finds every launch before its predecessor complete: the x-row
// kernel's RK stages use this to request their stage input (written by the x-row launch before the
// convolution) ahead of the wait. A successor that starts early waits the same way, so the stream
// order of all other memory accesses is unchanged.
__device__ __forceinline__ void pdl_wait_then_release() {
  asm volatile("griddepcontrol.wait;\n" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory");
}
template <class... P, class... A>
static void launch_pdl(void (*k)(P...), unsigned grid, unsigned block, size_t smem, cudaStream_t st, A&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, k, static_cast<A&&>(args)...);
}

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
