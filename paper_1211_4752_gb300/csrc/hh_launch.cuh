// Kernel launch with programmatic stream serialization (programmatic
// dependent launch): the kernel may start while the previous kernel on the
// stream finishes; it waits for that kernel with griddepcontrol.wait before
// touching its output (griddep_wait in hh_tma.cuh).
#pragma once
#include <cuda_runtime.h>

namespace hh {

template <typename... KArgs, typename... Args>
void launch_pdl(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, kern, static_cast<KArgs>(args)...);
}

// The same launch without the attribute (stream order as usual).
template <typename... KArgs, typename... Args>
void launch_plain(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                  Args... args) {
  kern<<<grid, block, smem, s>>>(static_cast<KArgs>(args)...);
}

}  // namespace hh
