// prims.cuh -- generic device primitives used by the libskim pipeline:
// exclusive scan and a stable LSD radix sort (key uint64, value uint32).
#pragma once
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

namespace skim {

// Exclusive prefix sum of n uint64 values (in may equal out).  If total is
// non-null the sum of all values is written there (device pointer).  Needs
// scan_workspace_bytes(n) bytes of device workspace.
size_t scan_workspace_bytes(size_t n);
cudaError_t exclusive_scan_u64(const uint64_t *in, uint64_t *out, size_t n, uint64_t *total,
                               void *ws, cudaStream_t s);

// Stable LSD radix sort of (keys, vals) by the low `bits` bits of the keys.
// The sorted result ends in keys/vals; alt_keys/alt_vals are scratch of the
// same size.  Needs radix_workspace_bytes(n) bytes of workspace.
size_t radix_workspace_bytes(size_t n);
cudaError_t radix_sort_pairs(uint64_t *keys, uint32_t *vals, uint64_t *alt_keys, uint32_t *alt_vals,
                             size_t n, int bits, void *ws, cudaStream_t s);

}  // namespace skim
