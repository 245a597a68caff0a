// Device kernels of the s-step enlarged CG path (sm_103a).
//
// Every n x w block of vectors is row-major (element (i, c) at [i*w + c]); a multi-block
// operand (MB) is `count` such blocks kept in a ring of equally spaced slots, so the basis
// window of s-step SRE-CG (Algorithm 4), the (s+1)t window of CA SRE-CG and the full history
// of SRE-CG2 / MSDO-CG (Algorithms 3, 6) all use the same descriptor.
//
// Reductions over the n rows (block inner products, Gram matrices, residual norms) are
// two-stage and deterministic: a fixed grid writes one partial per CTA, a second kernel sums
// the partials in CTA order.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace ekcg {

constexpr int kThreads = 256;
constexpr int kGramRows = 32;   // rows staged per step of the Gram kernel
constexpr int kGramTile = 64;   // output tile of the Gram kernel (kGramTile^2 per CTA)
constexpr int kUpdRows = 32;    // rows per step of the block-update kernel
constexpr int kPMax = 256;      // max contraction width of one block-update launch

template <typename T>
struct MB {
    T* base;         // slot 0
    int64_t stride;  // elements between consecutive slots
    int first;       // slot holding block 0
    int count;       // number of blocks
    int ring;        // number of slots in the ring
    int w;           // columns per block
    __host__ __device__ __forceinline__ T* blk(int i) const {
        return base + (int64_t)((first + i) % ring) * stride;
    }
    __host__ __device__ __forceinline__ int cols() const { return count * w; }
};

template <typename T>
__host__ __device__ inline MB<const T> as_const(const MB<T>& m) {
    return MB<const T>{m.base, m.stride, m.first, m.count, m.ring, m.w};
}

// Deterministic CTA-wide sum (fixed shuffle tree, then warp sums in warp order).
template <typename Acc>
__device__ __forceinline__ Acc block_sum(Acc v, Acc* red) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) red[wid] = v;
    __syncthreads();
    Acc s = 0;
    if (threadIdx.x == 0) {
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += red[i];
    }
    __syncthreads();
    return s;
}

// ---------------------------------------------------------------------------------------
// Permutations, splitting operator T (Section 2), residual
// ---------------------------------------------------------------------------------------

template <typename T>
__global__ void k_gather(T* __restrict__ y, const T* __restrict__ x,
                         const int32_t* __restrict__ perm, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        y[i] = x[perm[i]];
}

template <typename T>
__global__ void k_scatter(T* __restrict__ y, const T* __restrict__ x,
                          const int32_t* __restrict__ perm, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        y[perm[i]] = x[i];
}

// T(r): row i of the n x t block holds r_i in the column of its domain, zeros elsewhere.
template <typename T>
__global__ void k_split_T(T* __restrict__ out, const T* __restrict__ r,
                          const int32_t* __restrict__ dom, int64_t n, int t) {
    const int64_t total = n * t;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / t;
        const int c = (int)(e - i * t);
        out[e] = (c == dom[i]) ? r[i] : T(0);
    }
}

// r = b - A x (float64) and per-CTA partials of ||r||^2.
__global__ void k_residual(double* __restrict__ r, const double* __restrict__ b,
                           const double* __restrict__ x, const int32_t* __restrict__ rowptr,
                           const int32_t* __restrict__ col, const double* __restrict__ val,
                           int64_t n, double* __restrict__ partials) {
    __shared__ double red[32];
    double local = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        double acc = 0.0;
        for (int j = rowptr[i]; j < rowptr[i + 1]; ++j) acc += val[j] * x[col[j]];
        const double ri = b[i] - acc;
        r[i] = ri;
        local += ri * ri;
    }
    const double s = block_sum(local, red);
    if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

// out = sqrt(sum of partials), summed in CTA order.
__global__ void k_norm_finalize(const double* __restrict__ partials, int g,
                                double* __restrict__ out) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double s = 0.0;
        for (int i = 0; i < g; ++i) s += partials[i];
        out[0] = sqrt(s);
    }
}

// ---------------------------------------------------------------------------------------
// Sparse matrix x block of vectors: U = A W (CSR, one thread per output element)
// ---------------------------------------------------------------------------------------

template <typename T>
__global__ void k_spmm(T* __restrict__ U, const T* __restrict__ W,
                       const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                       const T* __restrict__ val, int64_t n, int w) {
    const int64_t total = n * w;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / w;
        const int c = (int)(e - i * w);
        T acc = T(0);
        const int j1 = rowptr[i + 1];
        for (int j = rowptr[i]; j < j1; ++j) acc += val[j] * W[(int64_t)col[j] * w + c];
        U[e] = acc;
    }
}

// Vectorised variant: each thread owns 16 bytes of an output row (4 floats or 2 doubles);
// threads of a row share the row's (col, val) loads through L1.  Needs w * sizeof(T) a
// multiple of 16 and 16-byte aligned W and U.
template <typename T>
struct Vec16;
template <>
struct Vec16<float> {
    using V = float4;
    static constexpr int N = 4;
    __device__ __forceinline__ static void fma(V& a, float s, const V& b) {
        a.x += s * b.x; a.y += s * b.y; a.z += s * b.z; a.w += s * b.w;
    }
    __device__ __forceinline__ static V zero() { return make_float4(0.f, 0.f, 0.f, 0.f); }
};
template <>
struct Vec16<double> {
    using V = double2;
    static constexpr int N = 2;
    __device__ __forceinline__ static void fma(V& a, double s, const V& b) {
        a.x += s * b.x; a.y += s * b.y;
    }
    __device__ __forceinline__ static V zero() { return make_double2(0.0, 0.0); }
};

template <typename T>
__global__ void __launch_bounds__(256)
k_spmm_vec(T* __restrict__ U, const T* __restrict__ W, const int32_t* __restrict__ rowptr,
           const int32_t* __restrict__ col, const T* __restrict__ val, int64_t n, int w) {
    using VT = Vec16<T>;
    using V = typename VT::V;
    const int nv = w / VT::N;                 // vectors per row
    const int64_t total = n * nv;
    const V* Wv = reinterpret_cast<const V*>(W);
    V* Uv = reinterpret_cast<V*>(U);
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / nv;
        const int c = (int)(e - i * nv);
        const int j0 = __ldg(rowptr + i), j1 = __ldg(rowptr + i + 1);
        V acc = VT::zero();
        int j = j0;
        for (; j + 4 <= j1; j += 4) {
            const int c0 = __ldg(col + j), c1 = __ldg(col + j + 1), c2 = __ldg(col + j + 2),
                      c3 = __ldg(col + j + 3);
            const T v0 = __ldg(val + j), v1 = __ldg(val + j + 1), v2 = __ldg(val + j + 2),
                    v3 = __ldg(val + j + 3);
            const V w0 = Wv[(int64_t)c0 * nv + c], w1 = Wv[(int64_t)c1 * nv + c],
                    w2 = Wv[(int64_t)c2 * nv + c], w3 = Wv[(int64_t)c3 * nv + c];
            VT::fma(acc, v0, w0);
            VT::fma(acc, v1, w1);
            VT::fma(acc, v2, w2);
            VT::fma(acc, v3, w3);
        }
        for (; j < j1; ++j) VT::fma(acc, __ldg(val + j), Wv[(int64_t)__ldg(col + j) * nv + c]);
        Uv[e] = acc;
    }
}

// ---------------------------------------------------------------------------------------
// Tall-skinny products C = X^T Y (Gram matrices, CGS coefficients, alpha = V^T r)
// ---------------------------------------------------------------------------------------

// Float-float accumulator: hi + lo carries about 48 significant bits.  add_prod adds the
// exact product a*b (the rounding error of the float product is recovered with an FMA)
// using TwoSum on the high part.
struct DF {
    float hi, lo;
};
__device__ __forceinline__ void df_add_prod(DF& acc, float a, float b) {
    const float p = a * b;
    const float e = fmaf(a, b, -p);
    const float s = acc.hi + p;
    const float v = s - acc.hi;
    const float err = (acc.hi - (s - v)) + (p - v);
    acc.hi = s;
    acc.lo += err + e;
}

// Accumulation policy of the Gram kernel: Acc = T (plain), double from float64 data, and
// float-float (stored as double) when float32 data must give a float64-grade Gram matrix.
template <typename T, typename Acc>
struct GramAcc {
    using R = Acc;
    __device__ __forceinline__ static void zero(R& a) { a = R(0); }
    __device__ __forceinline__ static void add(R& a, T x, T y) { a += (R)x * (R)y; }
    __device__ __forceinline__ static Acc out(const R& a) { return a; }
};
template <>
struct GramAcc<float, double> {
    using R = DF;
    __device__ __forceinline__ static void zero(R& a) { a.hi = 0.f; a.lo = 0.f; }
    __device__ __forceinline__ static void add(R& a, float x, float y) { df_add_prod(a, x, y); }
    __device__ __forceinline__ static double out(const R& a) {
        return (double)a.hi + (double)a.lo;
    }
};

// Stage rows [r0, r0 + kGramRows) x columns [c0, c0 + width) of a multi-block operand.
template <typename T, typename Acc, int LD>
__device__ __forceinline__ void stage_cols(Acc* dst, const MB<const T>& X, int64_t r0, int64_t n,
                                           int c0, int width) {
    const int P = X.cols();
    for (int e = threadIdx.x; e < kGramRows * width; e += blockDim.x) {
        const int rr = e / width, cc = e - rr * width;
        const int64_t row = r0 + rr;
        const int gc = c0 + cc;
        Acc v = Acc(0);
        if (row < n && gc < P) {
            const int b = gc / X.w;
            v = (Acc)X.blk(b)[row * X.w + (gc - b * X.w)];
        }
        dst[rr * LD + cc] = v;
    }
}

// Output tile (TPT*MP) x (TQT*MQ); TPT*TQT = kThreads threads, each an MP x MQ micro-tile.
// grid = (G row CTAs, tiles); partials[(tile*G + cta)*kGramTile^2 + i*TQ + j]
// (each tile's partials keep a kGramTile^2 stride whatever the tile shape).
template <typename T, typename Acc, int TPT, int TQT, int MP, int MQ>
__global__ void __launch_bounds__(kThreads)
k_gram_partial(MB<const T> X, MB<const T> Y, int64_t n, int ntq, Acc* __restrict__ partials) {
    constexpr int TP = TPT * MP, TQ = TQT * MQ;
    static_assert(TPT * TQT == kThreads, "thread layout");
    static_assert(TP * TQ <= kGramTile * kGramTile, "tile");
    using Pol = GramAcc<T, Acc>;
    __shared__ T xs[kGramRows * (TP + 1)];
    __shared__ T ys[kGramRows * (TQ + 1)];
    const int tile = blockIdx.y;
    const int p0 = (tile / ntq) * TP, q0 = (tile % ntq) * TQ;
    const int ti = threadIdx.x / TQT, tj = threadIdx.x % TQT;
    typename Pol::R acc[MP][MQ];
#pragma unroll
    for (int a = 0; a < MP; ++a)
#pragma unroll
        for (int c = 0; c < MQ; ++c) Pol::zero(acc[a][c]);
    for (int64_t r0 = (int64_t)blockIdx.x * kGramRows; r0 < n;
         r0 += (int64_t)gridDim.x * kGramRows) {
        stage_cols<T, T, TP + 1>(xs, X, r0, n, p0, TP);
        stage_cols<T, T, TQ + 1>(ys, Y, r0, n, q0, TQ);
        __syncthreads();
#pragma unroll 4
        for (int rr = 0; rr < kGramRows; ++rr) {
            T a[MP], bq[MQ];
#pragma unroll
            for (int k = 0; k < MP; ++k) a[k] = xs[rr * (TP + 1) + ti * MP + k];
#pragma unroll
            for (int k = 0; k < MQ; ++k) bq[k] = ys[rr * (TQ + 1) + tj * MQ + k];
#pragma unroll
            for (int k = 0; k < MP; ++k)
#pragma unroll
                for (int l = 0; l < MQ; ++l) Pol::add(acc[k][l], a[k], bq[l]);
        }
        __syncthreads();
    }
    Acc* out = partials + ((int64_t)tile * gridDim.x + blockIdx.x) * (kGramTile * kGramTile);
#pragma unroll
    for (int k = 0; k < MP; ++k)
#pragma unroll
        for (int l = 0; l < MQ; ++l)
            out[(ti * MP + k) * TQ + tj * MQ + l] = Pol::out(acc[k][l]);
}

// float32 Gram for HBM-bound shapes: every warp owns the whole P x Q output (lanes LP x LQ,
// micro-tile MP x MQ, P = LP*MP and Q = LQ*MQ exactly) and walks its own 32-row groups.
// Rows are double-buffered into the warp's shared-memory slice with cp.async (16-byte
// copies, no cross-warp waits), read back as float4, and the warps' tiles are summed in warp
// order at the end (deterministic).  Block widths must be multiples of 4 floats.
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;"); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;"); }
__device__ __forceinline__ void cp_async_wait0() { asm volatile("cp.async.wait_group 0;"); }

template <typename Acc, int LP, int LQ, int MP, int MQ>
__global__ void __launch_bounds__(128)
k_gram_warp_f32(MB<const float> X, MB<const float> Y, int64_t n, Acc* __restrict__ partials) {
    // W: shared row stride, padded to 4 floats so every 16-byte copy stays aligned
    constexpr int P = LP * MP, Q = LQ * MQ, W = (P + Q + 3) / 4 * 4, kWarps = 4, RG = 16;
    static_assert(P % 4 == 0, "X part of a staged row must be 16-byte aligned");
    static_assert(LP * LQ == 32, "one warp");
    using Pol = GramAcc<float, Acc>;
    extern __shared__ __align__(16) float gsm[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float* buf = gsm + warp * (2 * RG * W);        // [2][RG rows][P | Q]
    const int li = lane / LQ, lj = lane % LQ;
    typename Pol::R acc[MP][MQ];
#pragma unroll
    for (int a = 0; a < MP; ++a)
#pragma unroll
        for (int c = 0; c < MQ; ++c) Pol::zero(acc[a][c]);
    const int64_t groups = (n + RG - 1) / RG;
    const int64_t gw = (int64_t)gridDim.x * kWarps;
    int64_t g = (int64_t)blockIdx.x * kWarps + warp;
    // copies of row group gg into slot sl; rows past n are zero-filled
    auto stage_op = [&](const MB<const float>& M, int col0, int64_t r0, int rows, float* dst) {
        for (int b = 0; b < M.count; ++b) {
            const float* src = M.blk(b) + r0 * M.w;
            if (M.w % 4 == 0) {
                const int w4 = M.w / 4;
                for (int e = lane; e < RG * w4; e += 32) {
                    const int rr = e / w4, c4 = e - rr * w4;
                    float* d = dst + rr * W + col0 + b * M.w + c4 * 4;
                    if (rr < rows)
                        cp_async16(d, src + rr * M.w + c4 * 4);
                    else
                        *reinterpret_cast<float4*>(d) = make_float4(0.f, 0.f, 0.f, 0.f);
                }
            } else {
                for (int e = lane; e < RG * M.w; e += 32) {
                    const int rr = e / M.w, cc = e - rr * M.w;
                    float* d = dst + rr * W + col0 + b * M.w + cc;
                    if (rr < rows) {
                        const unsigned sa = (unsigned)__cvta_generic_to_shared(d);
                        asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(sa),
                                     "l"(src + rr * M.w + cc) : "memory");
                    } else {
                        *d = 0.f;
                    }
                }
            }
        }
    };
    auto issue = [&](int64_t gg, int sl) {
        float* dst = buf + sl * RG * W;
        const int64_t r0 = gg * RG;
        const int64_t rem = n - r0;
        const int rows = rem < RG ? (int)rem : RG;
        stage_op(X, 0, r0, rows, dst);
        stage_op(Y, P, r0, rows, dst);
    };
    int slot = 0;
    if (g < groups) issue(g, 0);
    cp_async_commit();
    for (; g < groups; g += gw) {
        const int64_t nx = g + gw;
        if (nx < groups) issue(nx, slot ^ 1);
        cp_async_commit();
        cp_async_wait1();
        __syncwarp();
        const float* cur = buf + slot * RG * W;
#pragma unroll 2
        for (int rr = 0; rr < RG; ++rr) {
            float a[MP], bq[MQ];
#pragma unroll
            for (int k = 0; k < MP; k += (MP % 4 == 0 ? 4 : 1)) {
                if (MP % 4 == 0) {
                    const float4 v = *reinterpret_cast<const float4*>(cur + rr * W + li * MP + k);
                    a[k] = v.x; a[k + 1] = v.y; a[k + 2] = v.z; a[k + 3] = v.w;
                } else {
                    a[k] = cur[rr * W + li * MP + k];
                }
            }
#pragma unroll
            for (int k = 0; k < MQ; k += (MQ % 4 == 0 ? 4 : 1)) {
                if (MQ % 4 == 0) {
                    const float4 v = *reinterpret_cast<const float4*>(cur + rr * W + P + lj * MQ + k);
                    bq[k] = v.x; bq[k + 1] = v.y; bq[k + 2] = v.z; bq[k + 3] = v.w;
                } else {
                    bq[k] = cur[rr * W + P + lj * MQ + k];
                }
            }
#pragma unroll
            for (int k = 0; k < MP; ++k)
#pragma unroll
                for (int l = 0; l < MQ; ++l) Pol::add(acc[k][l], a[k], bq[l]);
        }
        __syncwarp();
        slot ^= 1;
    }
    cp_async_wait0();
    __syncthreads();
    // warp tiles -> shared memory (reusing the staging space), summed in warp order
    Acc* red = reinterpret_cast<Acc*>(gsm);
#pragma unroll
    for (int k = 0; k < MP; ++k)
#pragma unroll
        for (int l = 0; l < MQ; ++l)
            red[warp * P * Q + (li * MP + k) * Q + lj * MQ + l] = Pol::out(acc[k][l]);
    __syncthreads();
    Acc* out = partials + (int64_t)blockIdx.x * (kGramTile * kGramTile);
    for (int e = threadIdx.x; e < P * Q; e += blockDim.x) {
        Acc s = Acc(0);
        for (int w = 0; w < kWarps; ++w) s += red[w * P * Q + e];
        out[e] = s;
    }
}

// Block times one vector, c = X^T r (the s-step coefficients alpha = V^T r): P <= 256
// columns of X, one right-hand column.  Thread (phase ph, column p) walks rows
// ph, ph + phases, ... of the CTA's row stripe: the P threads of a phase read one row of every
// block of X contiguously and r[row] by broadcast; eight rows are loaded before they are
// added.  The phases of a CTA are summed in phase order into its partial (partials[cta*4096
// + p]); k_gram_reduce then sums the CTAs in order.
template <typename T, typename Acc>
__global__ void __launch_bounds__(kThreads)
k_gram_vec(MB<const T> X, const T* __restrict__ r, int64_t n, Acc* __restrict__ partials) {
    __shared__ Acc red[kThreads];
    const int P = X.cols();
    const int phases = kThreads / P;
    const int tid = threadIdx.x;
    const bool active = tid < phases * P;
    const int p = active ? tid % P : 0, ph = active ? tid / P : 0;
    const int b = p / X.w, cc = p - b * X.w;
    const T* xb = X.blk(b);
    const int64_t stride = (int64_t)gridDim.x * phases;
    Acc acc = Acc(0);
    if (active) {
        int64_t row = (int64_t)blockIdx.x * phases + ph;
        for (; row + 7 * stride < n; row += 8 * stride) {
            T xv[8], rv[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                xv[u] = xb[(row + u * stride) * X.w + cc];
                rv[u] = r[row + u * stride];
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) acc += (Acc)xv[u] * (Acc)rv[u];
        }
        for (; row < n; row += stride) acc += (Acc)xb[row * X.w + cc] * (Acc)r[row];
    }
    red[tid] = acc;
    __syncthreads();
    for (int q = tid; q < P; q += kThreads) {
        Acc s = Acc(0);
        for (int h = 0; h < phases; ++h) s += red[h * P + q];
        partials[(int64_t)blockIdx.x * (kGramTile * kGramTile) + q] = s;
    }
}

// C[(c_row0 + p)*ldc + q] = sum over the g CTAs of the partials, p < P, q < Q.  One warp per
// output: lane l adds the partials of CTAs l, l + 32, ... in CTA order, and the 32 lane sums
// are combined by a fixed shuffle tree (the same order on every call).
template <typename Acc, typename Out>
__global__ void k_gram_reduce(const Acc* __restrict__ partials, int g, int ntq, int TP, int TQ,
                              int P, int Q, Out* __restrict__ C, int ldc, int c_row0) {
    const int total = P * Q;
    const int lane = threadIdx.x & 31;
    const int nwarps = (int)((gridDim.x * blockDim.x) >> 5);
    for (int e = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5); e < total; e += nwarps) {
        const int p = e / Q, q = e - p * Q;
        const int tile = (p / TP) * ntq + q / TQ;
        const int loc = (p % TP) * TQ + (q % TQ);
        const Acc* src = partials + (int64_t)tile * g * (kGramTile * kGramTile) + loc;
        Acc s = Acc(0);
        for (int c = lane; c < g; c += 32) s += src[(int64_t)c * (kGramTile * kGramTile)];
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) C[(int64_t)(c_row0 + p) * ldc + q] = (Out)s;
    }
}

// CTAs for k_gram_reduce: one warp per output, at most 4 CTAs per SM.
inline int reduce_grid(int outputs, int num_sms) {
    const int warps_per_cta = kThreads / 32;
    const int need = (outputs + warps_per_cta - 1) / warps_per_cta;
    return need < 1 ? 1 : (need < num_sms * 4 ? need : num_sms * 4);
}

// ---------------------------------------------------------------------------------------
// Block update: OUT = beta*Y + alpha * X C  (CGS step W - Q C, and W R^{-1})
// ---------------------------------------------------------------------------------------
// X has P <= kPMax columns; C is P x Q with leading dimension ldc starting at row c_row0.
// upper = 1 when C is upper triangular (only k <= q contributes).  OUT may alias X or Y:
// each CTA stages its kUpdRows rows of X in shared memory before writing any of them.
// Layout: lane = row of the tile, warp = group of 4 output columns, so the column-dependent
// trip count of the triangular case is uniform across a warp and the C values a warp reads
// are broadcasts.
template <typename T, typename CT>
__global__ void __launch_bounds__(kThreads)
k_update(MB<const T> X, const CT* __restrict__ C, int ldc, int c_row0, MB<const T> Y,
         MB<T> OUT, int64_t n, int beta_on, CT alpha, int upper) {
    static_assert(kUpdRows == 32, "one lane per row");
    extern __shared__ unsigned char smem_raw[];
    T* xs = reinterpret_cast<T*>(smem_raw);
    const int P = X.cols(), Q = OUT.cols();
    const int ldx = P + 1;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    const int ngroups = (Q + 3) >> 2;
    const CT* Cb = C + (int64_t)c_row0 * ldc;
    for (int64_t r0 = (int64_t)blockIdx.x * kUpdRows; r0 < n;
         r0 += (int64_t)gridDim.x * kUpdRows) {
        for (int e = threadIdx.x; e < kUpdRows * P; e += blockDim.x) {
            const int rr = e / P, cc = e - rr * P;
            const int64_t row = r0 + rr;
            const int b = cc / X.w;
            xs[rr * ldx + cc] = (row < n) ? X.blk(b)[row * X.w + (cc - b * X.w)] : T(0);
        }
        __syncthreads();
        const int64_t row = r0 + lane;
        const T* xr = xs + lane * ldx;
        for (int g = warp; g < ngroups; g += nwarp) {
            const int q0 = g * 4;
            const int nq = min(4, Q - q0);
            const int kend = upper ? min(P, q0 + 4) : P;
            CT acc0 = CT(0), acc1 = CT(0), acc2 = CT(0), acc3 = CT(0);
            if (nq == 4) {
                for (int k = 0; k < kend; ++k) {
                    const CT xv = (CT)xr[k];
                    const CT* cr = Cb + (int64_t)k * ldc + q0;
                    acc0 += xv * cr[0];
                    acc1 += xv * cr[1];
                    acc2 += xv * cr[2];
                    acc3 += xv * cr[3];
                }
            } else {
                for (int k = 0; k < kend; ++k) {
                    const CT xv = (CT)xr[k];
                    const CT* cr = Cb + (int64_t)k * ldc + q0;
                    acc0 += xv * cr[0];
                    if (nq > 1) acc1 += xv * cr[1];
                    if (nq > 2) acc2 += xv * cr[2];
                }
            }
            if (row < n) {
                const CT accs[4] = {acc0, acc1, acc2, acc3};
                for (int c = 0; c < nq; ++c) {
                    const int q = q0 + c;
                    const int bo = q / OUT.w, co = q - bo * OUT.w;
                    CT y = CT(0);
                    if (beta_on) {
                        const int by = q / Y.w;
                        y = (CT)Y.blk(by)[row * Y.w + (q - by * Y.w)];
                    }
                    OUT.blk(bo)[row * OUT.w + co] = (T)(y + alpha * accs[c]);
                }
            }
        }
        __syncthreads();
    }
}

// float32 block update for HBM-bound shapes: each thread owns one row and 4 consecutive
// output columns.  The Q/4 threads of a row read the row of X as the same float4 values
// (broadcast through L1), C (P x Q <= 64 x 32) sits in shared memory and is read as float4,
// and Y / OUT are read and written as float4 runs along the row (coalesced).  The
// triangular case runs the full loop over the zero part of C: the threads of a warp would
// wait for the longest one anyway.  P, Q and every block width are multiples of 4 (16-byte
// aligned rows).  OUT may alias Y (each thread reads its own float4 of Y before writing it);
// OUT aliasing X is not allowed here (rows of X are read by several threads).
template <int P>
__global__ void __launch_bounds__(256)
k_update_f32(MB<const float> X, const float* __restrict__ C, int ldc, int c_row0,
             MB<const float> Y, MB<float> OUT, int64_t n, int beta_on, float alpha, int upper) {
    constexpr int kMaxQ = 32;
    __shared__ __align__(16) float cs[P * kMaxQ];
    const int Q = OUT.cols();
    for (int e = threadIdx.x; e < P * Q; e += blockDim.x) {
        const int k = e / Q, q = e - k * Q;
        cs[k * kMaxQ + q] = C[(int64_t)(c_row0 + k) * ldc + q];
    }
    __syncthreads();
    const int nq4 = Q / 4;
    const int64_t total = n * nq4;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t row = e / nq4;
        const int q0 = (int)(e - row * nq4) * 4;
        float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int k = 0; k < P; k += 4) {
            const int b = k / X.w;
            const float4 xv = *reinterpret_cast<const float4*>(X.blk(b) + row * X.w + (k - b * X.w));
            const float xs[4] = {xv.x, xv.y, xv.z, xv.w};
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) {
                const float4 c = *reinterpret_cast<const float4*>(cs + (k + kk) * kMaxQ + q0);
                acc.x += xs[kk] * c.x;
                acc.y += xs[kk] * c.y;
                acc.z += xs[kk] * c.z;
                acc.w += xs[kk] * c.w;
            }
        }
        float4 y = make_float4(0.f, 0.f, 0.f, 0.f);
        if (beta_on) {
            const int by = q0 / Y.w;
            y = *reinterpret_cast<const float4*>(Y.blk(by) + row * Y.w + (q0 - by * Y.w));
        }
        const int bo = q0 / OUT.w;
        float4 o;
        o.x = y.x + alpha * acc.x;
        o.y = y.y + alpha * acc.y;
        o.z = y.z + alpha * acc.z;
        o.w = y.w + alpha * acc.w;
        *reinterpret_cast<float4*>(OUT.blk(bo) + row * OUT.w + (q0 - bo * OUT.w)) = o;
    }
    (void)upper;
}

// In-place triangular form W <- W R^{-1} (P = Q <= 32): the Q/4 threads of a row are
// consecutive lanes of one warp (32 is a multiple of Q/4), so each thread loads the whole
// row of X into registers, the warp synchronises, and only then writes its 4 outputs.  The
// loop runs over whole warps so that every lane reaches the __syncwarp.
template <int P>
__global__ void __launch_bounds__(256)
k_rmul_f32(MB<float> X, const float* __restrict__ R, int ldr, int64_t n) {
    __shared__ __align__(16) float cs[P * P];
    for (int e = threadIdx.x; e < P * P; e += blockDim.x) {
        const int k = e / P, q = e - k * P;
        cs[e] = R[(int64_t)k * ldr + q];
    }
    __syncthreads();
    constexpr int nq4 = P / 4;
    static_assert(32 % nq4 == 0, "a row's threads must share a warp");
    const int64_t total = n * nq4;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t span = (total + 31) / 32 * 32;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < span; e += stride) {
        const bool live = e < total;
        const int64_t row = live ? e / nq4 : 0;
        const int q0 = live ? (int)(e - row * nq4) * 4 : 0;
        float x[P];
        if (live) {
#pragma unroll
            for (int k = 0; k < P; k += 4) {
                const int b = k / X.w;
                const float4 v =
                    *reinterpret_cast<const float4*>(X.blk(b) + row * X.w + (k - b * X.w));
                x[k] = v.x; x[k + 1] = v.y; x[k + 2] = v.z; x[k + 3] = v.w;
            }
        }
        __syncwarp();
        if (live) {
            float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
            for (int k = 0; k < P; ++k) {
                const float4 c = *reinterpret_cast<const float4*>(cs + k * P + q0);
                acc.x += x[k] * c.x;
                acc.y += x[k] * c.y;
                acc.z += x[k] * c.z;
                acc.w += x[k] * c.w;
            }
            const int bo = q0 / X.w;
            *reinterpret_cast<float4*>(X.blk(bo) + row * X.w + (q0 - bo * X.w)) = acc;
        }
        __syncwarp();
    }
}

// ---------------------------------------------------------------------------------------
// Small dense Cholesky G = R^T R (upper, from the upper triangle of G) and R^{-1}
// ---------------------------------------------------------------------------------------
// One CTA.  Right-looking, same operation order as the oracle.  Breakdown rule:
// d_i <= tol*|G_ii| or non-finite sets bit 0 of *flag and leaves R = Rinv = I.
__global__ void k_chol_inv(const double* __restrict__ G, int m, double* __restrict__ S,
                           double* __restrict__ R, double* __restrict__ Rinv, double tol,
                           int* __restrict__ flag, int deflate, int* __restrict__ ndefl) {
    // deflate != 0: a finite pivot that fails the breakdown rule drops its column (row e_i^T
    // in R, no Schur update from it; row and column i of R^{-1} zero, so W R^{-1} has a zero
    // column i); a block whose columns are all dropped is a breakdown.
    __shared__ int bad;
    __shared__ int ndrop;
    __shared__ unsigned char dropped[kPMax];
    const int tid = threadIdx.x, nt = blockDim.x;
    for (int e = tid; e < m * m; e += nt) {
        const int i = e / m, j = e - i * m;
        S[e] = (j >= i) ? G[e] : 0.0;
        R[e] = 0.0;
        Rinv[e] = 0.0;
    }
    for (int i = tid; i < m; i += nt) dropped[i] = 0;
    if (tid == 0) {
        bad = (*flag) & 1;
        ndrop = 0;
    }
    __syncthreads();
    for (int i = 0; i < m && !bad; ++i) {
        if (tid == 0) {
            const double d = S[i * m + i];
            if (!(d > tol * fabs(G[i * m + i])) || !isfinite(d)) {
                if (deflate && isfinite(d)) {
                    R[i * m + i] = 1.0;
                    dropped[i] = 1;
                    ++ndrop;
                } else {
                    bad = 1;
                }
            } else {
                R[i * m + i] = sqrt(d);
            }
        }
        __syncthreads();
        if (bad) break;
        if (dropped[i]) continue;
        const double rii = R[i * m + i];
        for (int j = i + 1 + tid; j < m; j += nt) R[i * m + j] = S[i * m + j] / rii;
        __syncthreads();
        const int rem = m - i - 1;
        for (int e = tid; e < rem * rem; e += nt) {
            const int j = i + 1 + e / rem, l = i + 1 + e % rem;
            if (l >= j) S[j * m + l] -= R[i * m + j] * R[i * m + l];
        }
        __syncthreads();
    }
    if (tid == 0 && !bad && ndrop == m) bad = 1;   // every column dropped
    __syncthreads();
    if (bad) {
        for (int e = tid; e < m * m; e += nt) {
            const int i = e / m, j = e - i * m;
            R[e] = (i == j) ? 1.0 : 0.0;
            Rinv[e] = R[e];
        }
        if (tid == 0) atomicOr(flag, 1);
        return;
    }
    // R^{-1} by back substitution, one column per thread.
    for (int c = tid; c < m; c += nt) {
        for (int i = c; i >= 0; --i) {
            double s = (i == c) ? 1.0 : 0.0;
            for (int k = i + 1; k <= c; ++k) s -= R[i * m + k] * Rinv[k * m + c];
            Rinv[i * m + c] = s / R[i * m + i];
        }
    }
    if (ndrop) {
        __syncthreads();
        for (int e = tid; e < m * m; e += nt) {
            const int i = e / m, j = e - i * m;
            if (dropped[i] || dropped[j]) Rinv[e] = 0.0;
        }
        if (tid == 0) atomicAdd(ndefl, ndrop);
    }
}

// ---------------------------------------------------------------------------------------
// X <- X R^{-1} by forward substitution along every row (A-CholQR, Section 3.1): each row
// x of the result solves x R = w for the row w of X, R upper triangular.  Right-looking
// order: x_i = w_i * (1 / R_ii), then w_j -= x_i R_ij for j > i.  The reciprocal is the
// diagonal of the R^{-1} that k_chol_inv writes (the correctly rounded 1 / R_ii).  Solving
// the triangular system keeps the backward error of each row at the level of R's rounding;
// multiplying by an explicitly inverted R adds the error of the inverse, which grows with
// the condition number of R and costs A-orthogonality on ill-conditioned blocks.
// One thread per row; the CTA's rows are staged in shared memory (row stride ld = m or m+1,
// odd, so that a half-warp's float64 accesses fall in distinct banks).
// ---------------------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(128)
k_trsm_rows(MB<T> X, const double* __restrict__ R, const double* __restrict__ Rinv, int m,
            int64_t n) {
    extern __shared__ unsigned char smem_raw[];
    double* xs = reinterpret_cast<double*>(smem_raw);
    const int ld = m | 1;
    const int rows = blockDim.x;
    for (int64_t r0 = (int64_t)blockIdx.x * rows; r0 < n; r0 += (int64_t)gridDim.x * rows) {
        for (int e = threadIdx.x; e < rows * m; e += blockDim.x) {
            const int rr = e / m, cc = e - rr * m;
            const int64_t row = r0 + rr;
            const int b = cc / X.w;
            xs[rr * ld + cc] = (row < n) ? (double)X.blk(b)[row * X.w + (cc - b * X.w)] : 0.0;
        }
        __syncthreads();
        double* xr = xs + threadIdx.x * ld;
        for (int i = 0; i < m; ++i) {
            const double xi = xr[i] * __ldg(Rinv + (int64_t)i * m + i);
            xr[i] = xi;
            const double* Ri = R + (int64_t)i * m;
            for (int j = i + 1; j < m; ++j) xr[j] = fma(-xi, __ldg(Ri + j), xr[j]);
        }
        __syncthreads();
        for (int e = threadIdx.x; e < rows * m; e += blockDim.x) {
            const int rr = e / m, cc = e - rr * m;
            const int64_t row = r0 + rr;
            const int b = cc / X.w;
            if (row < n) X.blk(b)[row * X.w + (cc - b * X.w)] = (T)xs[rr * ld + cc];
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------------------
// x += V alpha, r -= (A V) alpha, partials of ||r||^2   (Algorithm 4 last three lines)
// ---------------------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(kThreads)
k_xr_update(T* __restrict__ x, T* __restrict__ r, MB<const T> V, MB<const T> Z,
            const double* __restrict__ alpha, int64_t n, double* __restrict__ partials,
            const int* __restrict__ flag) {
    __shared__ double red[32];
    const bool skip = (*flag) != 0;   // breakdown: keep the last complete iterate
    double local = 0.0;
    if (!skip) {
        const int w = V.w;
        for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
             i += (int64_t)gridDim.x * blockDim.x) {
            double sx = 0.0, sr = 0.0;
            for (int b = 0; b < V.count; ++b) {
                const T* vb = V.blk(b) + i * w;
                const T* zb = Z.blk(b) + i * w;
                const double* ab = alpha + b * w;
                for (int c = 0; c < w; ++c) {
                    sx += (double)vb[c] * ab[c];
                    sr += (double)zb[c] * ab[c];
                }
            }
            const T xi = (T)((double)x[i] + sx);
            const T ri = (T)((double)r[i] - sr);
            x[i] = xi;
            r[i] = ri;
            local += (double)ri * (double)ri;
        }
    }
    const double s = block_sum(local, red);
    if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

// float32 x/r update of the inner solve: x += V alpha, r -= (A V) alpha in float arithmetic
// (alpha rounded to float).  The w/4 consecutive threads of a row (w/4 a power of two <= 32,
// so they share a warp) each take one float4 of every block and combine their partial sums
// with shuffles in a fixed order; the row's first thread writes x and r and adds r^2
// (float64) to the CTA partial of ||r||^2.  The loop runs over whole warps so that every
// lane reaches the shuffles.  Skipped after a breakdown, like k_xr_update.
constexpr int kMaxAlpha = 1024;
__global__ void __launch_bounds__(kThreads)
k_xr_update_f32(float* __restrict__ x, float* __restrict__ r, MB<const float> V,
                MB<const float> Z, const double* __restrict__ alpha, int64_t n,
                double* __restrict__ partials, const int* __restrict__ flag) {
    __shared__ float al[kMaxAlpha];
    __shared__ double red[32];
    const int w = V.w, g4 = w / 4, m = V.count * w;
    for (int i = threadIdx.x; i < m; i += blockDim.x) al[i] = (float)alpha[i];
    __syncthreads();
    const bool skip = (*flag) != 0;
    double local = 0.0;
    if (!skip) {
        const int64_t total = n * g4;
        const int64_t span = (total + 31) / 32 * 32;
        const int64_t stride = (int64_t)gridDim.x * blockDim.x;
        for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < span; e += stride) {
            const bool live = e < total;
            const int64_t i = live ? e / g4 : 0;
            const int q = live ? (int)(e - i * g4) : 0;
            float sx = 0.f, sr = 0.f;
            if (live) {
                for (int b = 0; b < V.count; ++b) {
                    const float4 v = *reinterpret_cast<const float4*>(V.blk(b) + i * w + 4 * q);
                    const float4 z = *reinterpret_cast<const float4*>(Z.blk(b) + i * w + 4 * q);
                    const float* a = al + b * w + 4 * q;
                    sx += v.x * a[0];
                    sx += v.y * a[1];
                    sx += v.z * a[2];
                    sx += v.w * a[3];
                    sr += z.x * a[0];
                    sr += z.y * a[1];
                    sr += z.z * a[2];
                    sr += z.w * a[3];
                }
            }
            for (int o = g4 / 2; o > 0; o >>= 1) {
                sx += __shfl_xor_sync(0xffffffffu, sx, o);
                sr += __shfl_xor_sync(0xffffffffu, sr, o);
            }
            if (live && q == 0) {
                const float xi = x[i] + sx;
                const float ri = r[i] - sr;
                x[i] = xi;
                r[i] = ri;
                local += (double)ri * (double)ri;
            }
        }
    }
    const double s = block_sum(local, red);
    if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

// ---------------------------------------------------------------------------------------
// Mixed precision helpers (float64 <-> float32 with scaling)
// ---------------------------------------------------------------------------------------
__global__ void k_to_float_scaled(float* __restrict__ y, const double* __restrict__ x,
                                  const double* __restrict__ norm, int64_t n) {
    const double sc = norm[0] > 0.0 ? 1.0 / norm[0] : 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        y[i] = (float)(x[i] * sc);
}

__global__ void k_axpy_scaled(double* __restrict__ x, const float* __restrict__ d,
                              const double* __restrict__ norm, int64_t n) {
    const double sc = norm[0];
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        x[i] += sc * (double)d[i];
}

// ---------------------------------------------------------------------------------------
// Matrix values on a fixed pattern, adjoint gradients, 2D diffusion model (edge form)
// ---------------------------------------------------------------------------------------

// val[jp] = vnat[map[jp]] (permuted storage from the caller's natural CSR order).
__global__ void k_refresh_values(double* __restrict__ val, float* __restrict__ val32,
                                 const double* __restrict__ vnat, const int32_t* __restrict__ map,
                                 int64_t nnz) {
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < nnz;
         j += (int64_t)gridDim.x * blockDim.x) {
        const double v = vnat[map[j]];
        val[j] = v;
        val32[j] = (float)v;
    }
}

// dL/dA_ij = -lambda_i x_j on the sparsity pattern, written in the caller's CSR order.
// lambda and x are natural-order vectors.
__global__ void k_grad_A(double* __restrict__ dval, const double* __restrict__ lam,
                         const double* __restrict__ x, const int32_t* __restrict__ rowptr,
                         const int32_t* __restrict__ col, const int32_t* __restrict__ perm,
                         const int32_t* __restrict__ map, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const double li = lam[perm[i]];
        for (int j = rowptr[i]; j < rowptr[i + 1]; ++j)
            dval[map[j]] = -li * x[perm[col[j]]];
    }
}

// Edge weight a * 2 k_p k_q / (k_p + k_q) (harmonic mean), no contraction so that the
// value matches a plain evaluation of the same expression.
__device__ __forceinline__ double hm_weight(double a, double kp, double kq) {
    return __dmul_rn(a, __ddiv_rn(__dmul_rn(__dmul_rn(2.0, kp), kq), __dadd_rn(kp, kq)));
}

// Values of the 5-point edge-form diffusion matrix A(kappa), kappa = exp(log_kappa), in
// natural CSR order with sorted columns (node p = i + nx*j).  Diagonal = sum of the edge
// weights of p plus a*kappa_p per Dirichlet face, added x-axis first then y-axis.
__global__ void k_diffusion2d_values(double* __restrict__ val, const double* __restrict__ logk,
                                     const int32_t* __restrict__ rowptr, int nx, int ny,
                                     double ax, double ay) {
    const int64_t n = (int64_t)nx * ny;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n;
         p += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(p % nx), j = (int)(p / nx);
        const double kp = exp(logk[p]);
        double wxl = 0.0, wxr = 0.0, wyd = 0.0, wyu = 0.0;
        if (i > 0) wxl = hm_weight(ax, exp(logk[p - 1]), kp);
        if (i < nx - 1) wxr = hm_weight(ax, kp, exp(logk[p + 1]));
        if (j > 0) wyd = hm_weight(ay, exp(logk[p - nx]), kp);
        if (j < ny - 1) wyu = hm_weight(ay, kp, exp(logk[p + nx]));
        double d = 0.0;
        d = __dadd_rn(d, wxr);
        d = __dadd_rn(d, wxl);
        if (i == 0) d = __dadd_rn(d, __dmul_rn(ax, kp));
        if (i == nx - 1) d = __dadd_rn(d, __dmul_rn(ax, kp));
        d = __dadd_rn(d, wyu);
        d = __dadd_rn(d, wyd);
        if (j == 0) d = __dadd_rn(d, __dmul_rn(ay, kp));
        if (j == ny - 1) d = __dadd_rn(d, __dmul_rn(ay, kp));
        int o = rowptr[p];
        if (j > 0) val[o++] = -wyd;
        if (i > 0) val[o++] = -wxl;
        val[o++] = d;
        if (i < nx - 1) val[o++] = -wxr;
        if (j < ny - 1) val[o++] = -wyu;
    }
}

// dL/dlog(kappa_p) for L(x(kappa)), x = A(kappa)^{-1} b, lambda = A^{-1} dL/dx:
// dL/dw_e = -(lambda_p - lambda_q)(x_p - x_q) for an edge, -lambda_p x_p for a face;
// dw_e/dk_p = a * 2 k_q^2 / (k_p + k_q)^2, dw_face/dk_p = a; dk_p/dlog k_p = k_p.
__global__ void k_diffusion2d_grad_logk(double* __restrict__ g, const double* __restrict__ logk,
                                        const double* __restrict__ lam,
                                        const double* __restrict__ x, int nx, int ny, double ax,
                                        double ay) {
    const int64_t n = (int64_t)nx * ny;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n;
         p += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(p % nx), j = (int)(p / nx);
        const double kp = exp(logk[p]);
        const double lp = lam[p], xp = x[p];
        double acc = 0.0;
        const int64_t nb[4] = {p - 1, p + 1, p - nx, p + nx};
        const bool ok[4] = {i > 0, i < nx - 1, j > 0, j < ny - 1};
        const double a[4] = {ax, ax, ay, ay};
        for (int e = 0; e < 4; ++e) {
            if (ok[e]) {
                const int64_t q = nb[e];
                const double kq = exp(logk[q]);
                const double s = kp + kq;
                acc += a[e] * (2.0 * kq * kq / (s * s)) * (-(lp - lam[q]) * (xp - x[q]));
            } else {
                acc += a[e] * (-lp * xp);
            }
        }
        g[p] = kp * acc;
    }
}

template <typename T>
__global__ void k_fill(T* __restrict__ y, T v, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        y[i] = v;
}

}  // namespace ekcg
