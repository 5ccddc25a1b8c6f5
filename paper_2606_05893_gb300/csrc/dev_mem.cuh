// Device memory of the library. Every device buffer of a PIC or U-Net handle is
// taken and returned through these two functions: cudaMalloc / cudaFree, or the
// caller's allocator when one is set with pic_set_allocator (include/pic.h).
#pragma once
#include <cuda_runtime.h>

#include <cstddef>

namespace pic {
cudaError_t dev_malloc(void** p, size_t bytes);
cudaError_t dev_free(void* p);
template <class T>
inline cudaError_t dev_malloc(T** p, size_t bytes) {
  return dev_malloc(reinterpret_cast<void**>(p), bytes);
}
// live handles (PIC and U-Net) that hold memory from the current allocator
void dev_handle_opened();
void dev_handle_closed();
}  // namespace pic
