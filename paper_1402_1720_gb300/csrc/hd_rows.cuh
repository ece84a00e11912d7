// Rows of the hull-restricted system matrix: count (row_ptr[i + 1] = row
// length, row_ptr[0] = 0), in-place inclusive scan of row_ptr[1..n] (scratch
// of rows_scan_scratch(n) int64), and emit into cols at row_ptr[i].  The
// hull is given as bytes and, optionally, packed (rows_hull_words(V) words,
// voxel v at bit v & 31 of word v >> 5): with the packed form, when it fits,
// every block holds the hull in shared memory.
#pragma once

#include "hd_internal.cuh"

namespace hd {

int64_t rows_hull_words(int64_t V);
cudaError_t launch_rows_count(const Inputs &in, int64_t n, const GeomQ &g, const Cordic &cd,
                              const uint8_t *hull, const uint32_t *hull_bits, int64_t *row_ptr,
                              int sm_count, cudaStream_t s);
int64_t rows_scan_scratch(int64_t n);
cudaError_t launch_rows_scan(int64_t *a, int64_t n, int64_t *scratch, cudaStream_t s);
cudaError_t launch_rows_emit(const Inputs &in, int64_t n, const GeomQ &g, const Cordic &cd,
                             const uint8_t *hull, const uint32_t *hull_bits,
                             const int64_t *row_ptr, int32_t *cols, int sm_count, cudaStream_t s);

}  // namespace hd
