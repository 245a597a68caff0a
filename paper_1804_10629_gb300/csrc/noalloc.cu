// Allocation-free block inner product C = X^T Y.
//
// Same operation as ekcg_gram (the two-stage, deterministic tall-skinny Gram), for callers
// that cannot allocate device memory: code that runs while a stream is being captured into
// a CUDA graph (a cudaMalloc there is not a stream operation and breaks or is refused by the
// capture), and programs whose device memory is owned by another allocator or fixed at
// start-up (a framework's caching pool, a real-time loop that must not allocate after
// initialisation).  Such a caller has no context workspace to lend, so the per-CTA partial
// tiles live in a fixed file-scope device array instead.
//
// Limits: p, q <= 64 (one 64 x 64 output tile) and at most kNoAllocCTAs row CTAs, so the
// scratch array is kNoAllocCTAs * 64 * 64 doubles = 2 MiB, held by every GPU that loads the
// library until the process exits.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/ekcg.h"

namespace {

constexpr int kNaTile = 64;        // output tile (p, q <= 64)
constexpr int kNaRows = 32;        // rows staged per step
constexpr int kNaThreads = 256;    // 16 x 16 threads, 4 x 4 outputs each
constexpr int kNoAllocCTAs = 64;   // row CTAs (partials slots)
constexpr int kMaxDevices = 64;

// The scratch: one partial 64 x 64 tile per row CTA.  In host code this name is only a
// stand-in for the symbol; the kernels get its device address from cudaGetSymbolAddress.
static __device__ __align__(256) double g_noalloc_partials[kNoAllocCTAs * kNaTile * kNaTile];

std::mutex g_mu;
void* g_scratch[kMaxDevices] = {nullptr};

// Each CTA accumulates X^T Y over its rows and writes its whole 64 x 64 tile (zeros outside
// p x q), so the reduction never reads a value left by an earlier call.
__global__ void __launch_bounds__(kNaThreads)
k_na_partial(const double* __restrict__ X, int p, const double* __restrict__ Y, int q,
             int64_t n, double* __restrict__ partials) {
    __shared__ double xs[kNaRows][kNaTile + 1];
    __shared__ double ys[kNaRows][kNaTile + 1];
    const int ti = threadIdx.x / 16, tj = threadIdx.x % 16;
    double acc[4][4] = {};
    for (int64_t r0 = (int64_t)blockIdx.x * kNaRows; r0 < n; r0 += (int64_t)gridDim.x * kNaRows) {
        for (int e = threadIdx.x; e < kNaRows * kNaTile; e += blockDim.x) {
            const int rr = e / kNaTile, cc = e % kNaTile;
            const int64_t row = r0 + rr;
            xs[rr][cc] = (row < n && cc < p) ? X[row * p + cc] : 0.0;
            ys[rr][cc] = (row < n && cc < q) ? Y[row * q + cc] : 0.0;
        }
        __syncthreads();
        for (int rr = 0; rr < kNaRows; ++rr) {
            double a[4], b[4];
            for (int k = 0; k < 4; ++k) {
                a[k] = xs[rr][ti * 4 + k];
                b[k] = ys[rr][tj * 4 + k];
            }
            for (int k = 0; k < 4; ++k)
                for (int l = 0; l < 4; ++l) acc[k][l] += a[k] * b[l];
        }
        __syncthreads();
    }
    double* out = partials + (int64_t)blockIdx.x * (kNaTile * kNaTile);
    for (int k = 0; k < 4; ++k)
        for (int l = 0; l < 4; ++l) out[(ti * 4 + k) * kNaTile + tj * 4 + l] = acc[k][l];
}

// C[i*q + j] = sum over the g CTAs, in CTA order.
__global__ void k_na_reduce(const double* __restrict__ partials, int g, int p, int q,
                            double* __restrict__ C) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < p * q; e += gridDim.x * blockDim.x) {
        const int i = e / q, j = e % q;
        double s = 0.0;
        for (int c = 0; c < g; ++c) s += partials[(int64_t)c * (kNaTile * kNaTile) + i * kNaTile + j];
        C[e] = s;
    }
}

// Device address of the scratch for the current device, looked up once per device.
int scratch_for_current_device(double** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return EKCG_ECUDA;
    if (dev < 0 || dev >= kMaxDevices) return EKCG_EINVAL;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch[dev]) {
        void* ptr = nullptr;
        if (cudaGetSymbolAddress(&ptr, g_noalloc_partials) != cudaSuccess || !ptr)
            return EKCG_ECUDA;
        g_scratch[dev] = ptr;
    }
    *out = (double*)g_scratch[dev];
    return EKCG_OK;
}

}  // namespace

extern "C" {

int ekcg_gram_noalloc(int64_t n, const double* X, int p, const double* Y, int q, double* C,
                      void* stream) {
    // sizes beyond the fixed scratch (one 64 x 64 tile per CTA) are rejected
    if (n < 1 || !X || !Y || !C || p < 1 || q < 1 || p > kNaTile || q > kNaTile)
        return EKCG_EINVAL;
    double* scratch = nullptr;
    int rc = scratch_for_current_device(&scratch);
    if (rc != EKCG_OK) return rc;
    const int64_t tiles = (n + kNaRows - 1) / kNaRows;
    const int g = (int)(tiles < kNoAllocCTAs ? tiles : kNoAllocCTAs);
    cudaStream_t st = (cudaStream_t)stream;
    k_na_partial<<<g, kNaThreads, 0, st>>>(X, p, Y, q, n, scratch);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) {
        const int gr = (p * q + 255) / 256;
        k_na_reduce<<<gr, 256, 0, st>>>(scratch, g, p, q, C);
        e = cudaGetLastError();
    }
    return e == cudaSuccess ? EKCG_OK : EKCG_ECUDA;
}

}  // extern "C"
