// rtalloc.h -- the host runtime's device and page-locked host allocations.
//
// Every allocation and free of the handle runtime (single boxes, ensembles,
// the D2Q9 handle, the closure's training scratch) goes through these
// wrappers.  They keep a count of live allocations and can be told to make one
// of the next allocations fail as if the device were out of memory
// (fpclbm_test_alloc_hook), so that tests can check on the host that every
// FPCLBM_ERR_ALLOC path frees what it had allocated and leaves the library
// usable.  A failed allocation sets the pointer to NULL.
#pragma once
#include <cuda_runtime.h>
#include <cstddef>

namespace fpc {

cudaError_t rt_malloc_raw(void** p, size_t bytes, bool host);
void rt_free_raw(void* p, bool host);

template <typename T>
cudaError_t rt_malloc(T** p, size_t bytes)
{
    void* v = nullptr;
    const cudaError_t e = rt_malloc_raw(&v, bytes, false);
    *p = static_cast<T*>(v);
    return e;
}

template <typename T>
cudaError_t rt_malloc_host(T** p, size_t bytes)
{
    void* v = nullptr;
    const cudaError_t e = rt_malloc_raw(&v, bytes, true);
    *p = static_cast<T*>(v);
    return e;
}

inline void rt_free(const void* p) { rt_free_raw(const_cast<void*>(p), false); }
inline void rt_free_host(const void* p) { rt_free_raw(const_cast<void*>(p), true); }

}  // namespace fpc
