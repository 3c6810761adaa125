#include "scan.cuh"

namespace nnqp {

namespace {

// Scan of one chunk per block; writes the inclusive-exclusive result and
// the chunk total.
__global__ void __launch_bounds__(kScanThreads) k_scan_chunks(const int64_t *in, int64_t *out, int64_t n,
                                                               int64_t *totals) {
    __shared__ int64_t warp_tot[kScanThreads / 32];
    const int64_t base = (int64_t)blockIdx.x * kScanChunk + (int64_t)threadIdx.x * kScanItems;
    int64_t v[kScanItems];
    int64_t run = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        int64_t x = base + k < n ? in[base + k] : 0;
        v[k] = run;
        run += x;
    }
    // exclusive scan of the per-thread totals across the block
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int64_t incl = run;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int64_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) warp_tot[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        int64_t t = lane < kScanThreads / 32 ? warp_tot[lane] : 0;
        int64_t ti = t;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int64_t y = __shfl_up_sync(0xffffffffu, ti, o);
            if (lane >= o) ti += y;
        }
        if (lane < kScanThreads / 32) warp_tot[lane] = ti - t;
        if (lane == kScanThreads / 32 - 1) totals[blockIdx.x] = ti;
    }
    __syncthreads();
    const int64_t off = warp_tot[warp] + incl - run;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k)
        if (base + k < n) out[base + k] = off + v[k];
}

__global__ void k_scan_add(int64_t *out, int64_t n, const int64_t *offs) {
    const int64_t base = (int64_t)blockIdx.x * kScanChunk;
    const int64_t o = offs[blockIdx.x];
    for (int64_t i = base + threadIdx.x; i < base + kScanChunk && i < n; i += blockDim.x) out[i] += o;
}

__global__ void k_set_total(int64_t *out, int64_t n, const int64_t *scanned_totals, int64_t nb) {
    out[n] = scanned_totals[nb];
}

}  // namespace

size_t scan_tmp_elems(int64_t n) {
    size_t s = 0;
    while (n > 1) {
        int64_t nb = (n + kScanChunk - 1) / kScanChunk;
        s += (size_t)(2 * nb + 2);
        n = nb;
    }
    return s + 4;
}

cudaError_t exclusive_scan(const int64_t *in, int64_t *out, int64_t n, int64_t *tmp, cudaStream_t st) {
    if (n == 0) {
        return cudaMemsetAsync(out, 0, sizeof(int64_t), st);
    }
    int64_t nb = (n + kScanChunk - 1) / kScanChunk;
    int64_t *totals = tmp;              // [nb]
    int64_t *tscan = tmp + nb;          // [nb + 1]
    (k_scan_chunks<<<(unsigned)nb, kScanThreads, 0, st>>>(in, out, n, totals), ::nnqp::count_launch());
    if (nb == 1) {
        (k_set_total<<<1, 1, 0, st>>>(out, n, totals, 0), ::nnqp::count_launch());  // out[n] = totals[0]
        return cudaGetLastError();
    }
    cudaError_t e = exclusive_scan(totals, tscan, nb, tmp + 2 * nb + 1, st);
    if (e != cudaSuccess) return e;
    (k_scan_add<<<(unsigned)nb, kScanThreads, 0, st>>>(out, n, tscan), ::nnqp::count_launch());
    (k_set_total<<<1, 1, 0, st>>>(out, n, tscan, nb), ::nnqp::count_launch());
    return cudaGetLastError();
}

namespace {

constexpr int kRedBlocks = 512;  // tmp must hold this many doubles
constexpr int kRedThreads = 256;

// MODE 0: sum, 1: sum of squares, 2: max
template <int MODE>
__device__ __forceinline__ double red_op(double a, double b) {
    return MODE == 2 ? fmax(a, b) : a + b;
}

template <int MODE>
__global__ void __launch_bounds__(kRedThreads) k_partial(const double *x, int64_t n, double *part) {
    __shared__ double sm[kRedThreads / 32];
    const int64_t per = (n + gridDim.x - 1) / gridDim.x;
    int64_t b0 = per * blockIdx.x, b1 = b0 + per;
    if (b0 > n) b0 = n;
    if (b1 > n) b1 = n;
    double s = MODE == 2 ? -INFINITY : 0.0;
    for (int64_t i = b0 + threadIdx.x; i < b1; i += blockDim.x) s = red_op<MODE>(s, MODE == 1 ? x[i] * x[i] : x[i]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s = red_op<MODE>(s, __shfl_xor_sync(0xffffffffu, s, o));
    if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = sm[0];
        for (int w = 1; w < kRedThreads / 32; ++w) t = red_op<MODE>(t, sm[w]);
        part[blockIdx.x] = t;
    }
}

template <int MODE>
__global__ void k_final(const double *part, int nb, double *out) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double t = part[0];
        for (int b = 1; b < nb; ++b) t = red_op<MODE>(t, part[b]);
        *out = t;
    }
}

}  // namespace

template <int MODE>
static cudaError_t det_reduce(const double *x, int64_t n, double *out, double *tmp, cudaStream_t st) {
    (k_partial<MODE><<<kRedBlocks, kRedThreads, 0, st>>>(x, n, tmp), ::nnqp::count_launch());
    (k_final<MODE><<<1, 32, 0, st>>>(tmp, kRedBlocks, out), ::nnqp::count_launch());
    return cudaGetLastError();
}

cudaError_t det_sum(const double *x, int64_t n, double *out, double *tmp, cudaStream_t st) {
    return det_reduce<0>(x, n, out, tmp, st);
}
cudaError_t det_sumsq(const double *x, int64_t n, double *out, double *tmp, cudaStream_t st) {
    return det_reduce<1>(x, n, out, tmp, st);
}
cudaError_t det_max(const double *x, int64_t n, double *out, double *tmp, cudaStream_t st) {
    return det_reduce<2>(x, n, out, tmp, st);
}

}  // namespace nnqp
