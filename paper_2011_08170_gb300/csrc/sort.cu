// Radix sort of (key, value) pairs for the create-time spatial renumbering.
// A library primitive (CUB, shipped with the CUDA toolkit); off the per-sweep path.
#include <cub/cub.cuh>

#include "f2m_internal.h"

namespace f2m {

cudaError_t sort_pairs_u64(void* temp, size_t& temp_bytes, const uint64_t* keys_in,
                           uint64_t* keys_out, const int32_t* vals_in, int32_t* vals_out,
                           int32_t count, int end_bit, cudaStream_t st) {
  return cub::DeviceRadixSort::SortPairs(temp, temp_bytes, keys_in, keys_out, vals_in, vals_out,
                                         count, 0, end_bit, st);
}

}  // namespace f2m
