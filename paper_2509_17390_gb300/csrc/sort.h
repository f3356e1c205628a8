// Device-wide exclusive scans and a stable LSD radix sort (sort.cu).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cstddef>

namespace fgl {

// Scratch elements an exclusive scan of n values needs (all levels of block sums).
size_t scan_tmp_elems(int64_t n);

// Exclusive prefix sums in place on `stream`; `tmp` holds scan_tmp_elems(n)
// elements.  `launches` counts the kernels launched.
cudaError_t scan_exclusive_u32(uint32_t* x, int64_t n, uint32_t* tmp, size_t tmp_elems,
                               cudaStream_t s, int* launches);
cudaError_t scan_exclusive_u64(unsigned long long* x, int64_t n, unsigned long long* tmp,
                               size_t tmp_elems, cudaStream_t s, int* launches);

// Scratch elements (uint32) of radix_sort_pairs over n pairs.
size_t radix_sort_tmp_elems(int64_t n);

// Stable sort of n (key, value) pairs by the low `bits` bits of the key, 8
// bits per pass, ping-ponging between (k0, v0) and (k1, v1); on return the
// sorted pairs are in the second buffers when *in_second, else in the first.
// Equal keys keep their input order.  n < 2^31.
cudaError_t radix_sort_pairs(uint32_t* k0, uint32_t* v0, uint32_t* k1, uint32_t* v1, int64_t n,
                             int bits, uint32_t* tmp, cudaStream_t s, int* launches,
                             bool* in_second);

}  // namespace fgl
