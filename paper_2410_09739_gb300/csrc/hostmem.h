// hostmem.h -- host-buffer helpers shared by the single-box and D2Q9 handles.
#pragma once
#include <cuda_runtime.h>

namespace fpc {

// Device address of host memory that the GPU can access directly: page-locked
// memory mapped into the device's address space (cudaHostAlloc, cudaHostRegister,
// pinned framework buffers).  nullptr for ordinary pageable memory, which goes
// through a device staging buffer instead.  With a mapped address the init and
// moments kernels read or write the caller's buffer in place over the host
// link, with no separate copy.
template <typename T>
T* mapped_host(T* p)
{
    if (!p) return nullptr;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    if (a.type != cudaMemoryTypeHost || !a.devicePointer) return nullptr;
    return static_cast<T*>(a.devicePointer);
}

}  // namespace fpc
