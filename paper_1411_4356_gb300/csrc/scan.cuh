#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace omss {
// rowptr[0..N] = exclusive prefix sums of counts[0..N-1]; scratch holds
// scan_scratch_size(N) int64 values.
void exclusive_scan_counts(const int64_t *counts, int64_t *rowptr, int64_t N, int64_t *scratch,
                           cudaStream_t s);
int64_t scan_scratch_size(int64_t N);
}  // namespace omss
