// Device-wide exclusive prefix sum of int64 counts and deterministic
// reductions (fixed block partition + fixed-order final pass).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace nnqp {

// Counts kernel launches made by the library (nn_kernel_launches).
void count_launch();

constexpr int kScanThreads = 512;
constexpr int kScanItems = 4;
constexpr int kScanChunk = kScanThreads * kScanItems;

// out[0..n] = exclusive scan of in[0..n-1]; out[n] = total.  Uses tmp of at
// least scan_tmp_elems(n) int64s.  Stream-ordered.
size_t scan_tmp_elems(int64_t n);
cudaError_t exclusive_scan(const int64_t *in, int64_t *out, int64_t n, int64_t *tmp, cudaStream_t st);

// Deterministic sum / max of a double array into *out (device).
cudaError_t det_sum(const double *x, int64_t n, double *out, double *tmp /*>= 1024*/, cudaStream_t st);
cudaError_t det_sumsq(const double *x, int64_t n, double *out, double *tmp, cudaStream_t st);
cudaError_t det_max(const double *x, int64_t n, double *out, double *tmp, cudaStream_t st);

}  // namespace nnqp
