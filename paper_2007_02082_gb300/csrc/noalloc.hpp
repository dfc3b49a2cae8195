// Canonical-order read of a parked state snapshot without device allocation
// (noalloc.cu).  The scratch is a fixed array of this module's device memory.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>

#include "ib.h"

namespace ibg {

// Capacity of the scratch in doubles (8 MiB): a field of nc * N values fits
// when nc * N <= NOALLOC_MAX_VALUES.
constexpr int64_t NOALLOC_MAX_VALUES = int64_t(1) << 20;

// Gather nc components of src (component c at src[c * nslots + canon[i]]) into
// canonical order, value (i, c) at position i * nc + c, through the scratch,
// and copy the bytes = nc * N * 8 result to dst (device memory when
// dst_on_device != 0, else host memory).  Synchronises st before returning.
ib_status noalloc_gather_canon(int64_t N, const int32_t* canon, int nc, int64_t nslots, const double* src,
                               void* dst, size_t bytes, int dst_on_device, cudaStream_t st, std::string& err);

}  // namespace ibg
