// Float32 block updates staged by the Tensor Memory Accelerator (bulk copies).
//
// OUT = Y + alpha X C for the CGS updates (X: the window blocks, P = nb * Q columns) and,
// with X = OUT, beta off and C = R^{-1}, the in-place A-CholQR product W <- W R^{-1}.  A
// persistent CTA walks row tiles of TR rows.  One thread issues, per tile, cp.async.bulk
// copies of the tile's rows of every block of X and of Y (a run of rows of a row-major
// n x Q block is contiguous), all completing on the stage's mbarrier; three stages keep two
// tiles in flight while the CTA computes the third.  Every thread then computes 4 rows x 4
// columns of the tile from shared memory (C sits in shared memory for the whole launch),
// reading each X value once per 4 output columns.  The sum over k runs in increasing k with
// one fused multiply-add per term, as in the unstaged kernel.
//
// Bank layout: a warp's lanes are kCG column groups x kG row groups, and the kG row groups
// read the same column of different rows at once.  Rows are 64 or 128 bytes long, so rows of
// one contiguous tile would all start in the same banks (a kG-way conflict on every X load).
// Each block's tile is therefore copied as kG sub-tiles of kSub rows, row group g taking its
// rows from sub-tile g, and sub-tile j is placed 16 j bytes further into shared memory than
// a dense layout would put it: the row groups' reads then fall into distinct 16-byte bank
// groups.
//
// Requirements (checked by the host before it picks this kernel): every block base and the
// slot stride 16-byte aligned, X.w == Q, Y and OUT single blocks, X not aliasing OUT unless
// it is the in-place product (then the tile is read completely before it is overwritten).
//
// Waits are bounded: if a stage does not complete within about 2^32 SM cycles the CTA sets
// bit 2 of *err, waits (again bounded) for the copies it has in flight and returns.
#pragma once

#include <cstdint>

#include "kernels.cuh"

namespace ekcg {
namespace bulk {

constexpr int kThreads = 256;
constexpr int kStages = 3;
constexpr long long kWaitCycles = 1ll << 32;

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
                 : "memory");
}
// make the initialised barriers visible to the bulk-copy (async) proxy
__device__ __forceinline__ void fence_barrier_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
                 "r"(bytes)
                 : "memory");
}
// global -> shared bulk copy (dst, src 16-byte aligned; bytes a multiple of 16)
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes,
                                         uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
            "r"(smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}
__device__ __forceinline__ bool mbar_test(uint64_t* bar, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return done != 0;
}
// true once the phase with this parity has completed; false after about `limit` cycles
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity,
                                          long long limit = kWaitCycles) {
    const long long t0 = clock64();
    while (!mbar_test(bar, parity))
        if (clock64() - t0 > limit) return false;
    return true;
}

// Diagnostic of the bounded wait: thread 0 arms an mbarrier for 16 bytes that no copy will
// deliver, every thread waits at most `limit` cycles, and the CTA sets bit 2 of *err when
// the wait runs out, the path the staged kernels take on a stage that never completes.
__global__ void k_wait_selftest(long long limit, int* err) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_barrier_init();
    }
    __syncthreads();
    if (threadIdx.x == 0) mbar_expect_tx(&bar, 16);
    __syncthreads();
    const bool ok = mbar_wait(&bar, 0, limit);
    if (__syncthreads_or(!ok) && threadIdx.x == 0) atomicOr(err, 4);
}

template <int P, int Q>
struct Shape {
    static_assert((Q == 16 || Q == 32) && P % Q == 0 && P <= 64, "bulk update shape");
    static constexpr int kCG = Q / 4;                    // float4 column groups
    static constexpr int kG = 32 / kCG;                  // row groups per warp
    static constexpr int kTR = 4 * kThreads / kCG;       // rows per tile (4 per thread)
    static constexpr int kSub = kTR / kG;                // rows per sub-tile (4 per warp)
    static constexpr int kSubF = kSub * Q + 4;           // floats per sub-tile, with the skew
    static constexpr int kSF = (P / Q + 1) * kG * kSubF; // floats per stage (X blocks, Y)
    static constexpr size_t kSmem = (size_t)(P * Q + kStages * kSF) * sizeof(float);
};

template <int P, int Q>
__global__ void __launch_bounds__(kThreads)
k_update_bulk_f32(MB<const float> X, const float* __restrict__ C, int ldc, int c_row0,
                  MB<const float> Y, MB<float> OUT, int64_t n, int beta_on, float alpha,
                  int* err) {
    using S = Shape<P, Q>;
    constexpr int NB = P / Q, TR = S::kTR, G = S::kG, SUB = S::kSub;
    extern __shared__ __align__(128) float sm[];
    __shared__ __align__(8) uint64_t full[kStages];
    float* cs = sm;                         // C: P x Q
    float* stage0 = sm + P * Q;             // kStages x (X tile blocks, Y tile)
    const int tid = threadIdx.x;
    const int64_t ntile = (n + TR - 1) / TR;
    const int64_t step = gridDim.x;

    auto issue = [&](int64_t tile, int st) {
        const int64_t row0 = tile * TR;
        const int rows = (int)((n - row0) < TR ? (n - row0) : TR);
        float* xs = stage0 + st * S::kSF;
        mbar_expect_tx(&full[st], (uint32_t)rows * Q * sizeof(float) * (NB + (beta_on ? 1 : 0)));
        for (int g = 0; g < G && g * SUB < rows; ++g) {
            const int r0 = g * SUB;
            const int nr = rows - r0 < SUB ? rows - r0 : SUB;
            const uint32_t bytes = (uint32_t)nr * Q * sizeof(float);
#pragma unroll
            for (int b = 0; b < NB; ++b)
                bulk_g2s(xs + (b * G + g) * S::kSubF, X.blk(b) + (row0 + r0) * Q, bytes,
                         &full[st]);
            if (beta_on)
                bulk_g2s(xs + (NB * G + g) * S::kSubF, Y.blk(0) + (row0 + r0) * Q, bytes,
                         &full[st]);
        }
    };

    if (tid == 0) {
        for (int s = 0; s < kStages; ++s) mbar_init(&full[s], 1);
        fence_barrier_init();
    }
    for (int e = tid; e < P * Q; e += kThreads) {
        const int k = e / Q, q = e - k * Q;
        cs[e] = C[(int64_t)(c_row0 + k) * ldc + q];
    }
    __syncthreads();
    int64_t issued = 0;   // tiles of this CTA whose copies have been issued
    if (tid == 0)
        for (int s = 0; s < kStages && blockIdx.x + s * step < ntile; ++s) issue(blockIdx.x + s * step, s);
    {
        int64_t c = 0;
        for (int s = 0; s < kStages && blockIdx.x + s * step < ntile; ++s) ++c;
        issued = c;
    }
    // lane = (row group g, column group cg); thread rows g * SUB + 4 warp + i, i < 4
    const int lane = tid & 31, warp = tid >> 5;
    const int cg = lane % S::kCG, g = lane / S::kCG;
    const int rloc = 4 * warp;             // first row of this thread within its sub-tile
    float* out = OUT.blk(0);
    int64_t it = 0;
    for (int64_t tile = blockIdx.x; tile < ntile; tile += step, ++it) {
        const int st = (int)(it % kStages);
        const bool ok = mbar_wait(&full[st], (uint32_t)((it / kStages) & 1));
        if (__syncthreads_or(!ok)) {
            if (tid == 0) {
                atomicOr(err, 4);
                for (int64_t j = it; j < issued; ++j)
                    (void)mbar_wait(&full[j % kStages], (uint32_t)((j / kStages) & 1));
            }
            __syncthreads();
            return;
        }
        const float* xs = stage0 + st * S::kSF + g * S::kSubF;   // this row group's sub-tiles
        const float* ys = stage0 + st * S::kSF + (NB * G + g) * S::kSubF;
        const int64_t row0 = tile * TR;
        float4 acc[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) acc[i] = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int k = 0; k < P; k += 4) {
            const int b = k / Q, kk = k - b * Q;
            float4 xv[4];
#pragma unroll
            for (int i = 0; i < 4; ++i)
                xv[i] = *reinterpret_cast<const float4*>(xs + b * G * S::kSubF + (rloc + i) * Q + kk);
            float4 c4[4];
#pragma unroll
            for (int j = 0; j < 4; ++j)
                c4[j] = *reinterpret_cast<const float4*>(cs + (k + j) * Q + cg * 4);
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const float xk[4] = {xv[i].x, xv[i].y, xv[i].z, xv[i].w};
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    acc[i].x += xk[j] * c4[j].x;
                    acc[i].y += xk[j] * c4[j].y;
                    acc[i].z += xk[j] * c4[j].z;
                    acc[i].w += xk[j] * c4[j].w;
                }
            }
        }
        const int rows = (int)((n - row0) < TR ? (n - row0) : TR);
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int r = g * SUB + rloc + i;
            if (r < rows) {
                float4 y = make_float4(0.f, 0.f, 0.f, 0.f);
                if (beta_on) y = *reinterpret_cast<const float4*>(ys + (rloc + i) * Q + cg * 4);
                float4 o;
                o.x = y.x + alpha * acc[i].x;
                o.y = y.y + alpha * acc[i].y;
                o.z = y.z + alpha * acc[i].z;
                o.w = y.w + alpha * acc[i].w;
                *reinterpret_cast<float4*>(out + (row0 + r) * Q + cg * 4) = o;
            }
        }
        __syncthreads();   // every thread is done with this stage
        if (tid == 0) {
            const int64_t next = tile + kStages * step;
            if (next < ntile) {
                issue(next, st);
                ++issued;
            }
        }
        // `issued` is only read by thread 0 (failure path)
    }
}

// ---------------------------------------------------------------------------------------
// Upper triangle of a Gram matrix G = X^T Y (X, Y: single n x M blocks, M = 16 or 32): the
// A-CholQR Gram W^T (A W) and the Pre-CholQR Gram W^T W, whose Cholesky factorisation reads
// only the entries i <= j.  G is cut into 4 x 8 lane blocks; the blocks that hold an entry
// on or above the diagonal (20 of 32 for M = 32, 6 of 8 for M = 16) are dealt to the 128
// threads of a CTA, each block to kPh threads that take every kPh-th row of a tile.  float
// data: exact float products added to float-float accumulators (df_add_prod, about 48
// significant bits); float64 data: float64 fused multiply-adds.  Row tiles are staged with
// bulk copies on the same three-stage mbarrier pipeline as the update.  At the end the kPh
// row phases are summed in phase order in double, and the CTA writes its M x M partial
// (zero below the computed blocks) for k_gram_reduce, which sums the CTAs in order.
// ---------------------------------------------------------------------------------------
constexpr int kUThreads = 128;

__host__ __device__ constexpr bool upper_block(int bi, int bj) { return 8 * bj + 7 >= 4 * bi; }
__host__ __device__ constexpr int upper_blocks(int M) {
    int c = 0;
    for (int bj = 0; bj < M / 8; ++bj)
        for (int bi = 0; bi < M / 4; ++bi)
            if (upper_block(bi, bj)) ++c;
    return c;
}

template <typename T, int M>
struct UpperShape {
    static_assert(M == 16 || M == 32, "upper Gram width");
    static constexpr int kNBlk = upper_blocks(M);
    static constexpr int kPh = kUThreads / kNBlk;        // threads per lane block (row phases)
    static constexpr int kTR = sizeof(T) == 4 ? 128 : 64;   // rows per tile
    static constexpr int kSF = 2 * kTR * M;              // elements per stage (X tile, Y tile)
    static constexpr size_t kStageBytes = (size_t)kStages * kSF * sizeof(T);
    static constexpr size_t kRedBytes = (size_t)kPh * kNBlk * 32 * sizeof(double);
    static constexpr size_t kSmem = kStageBytes > kRedBytes ? kStageBytes : kRedBytes;
};

template <typename T>
__device__ __forceinline__ void load4(const T* p, T* v) {
    if constexpr (sizeof(T) == 4) {
        const float4 q = *reinterpret_cast<const float4*>(p);
        v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
    } else {
        const double2 q0 = *reinterpret_cast<const double2*>(p);
        const double2 q1 = *reinterpret_cast<const double2*>(p + 2);
        v[0] = q0.x; v[1] = q0.y; v[2] = q1.x; v[3] = q1.y;
    }
}

template <typename T, int M>
__global__ void __launch_bounds__(kUThreads)
k_gram_upper(const T* __restrict__ X, const T* __restrict__ Y, int64_t n,
             double* __restrict__ partials, int* err) {
    using U = UpperShape<T, M>;
    using Pol = GramAcc<T, double>;
    constexpr int TR = U::kTR, NB = U::kNBlk, PH = U::kPh;
    extern __shared__ __align__(128) unsigned char smraw[];
    T* sm = reinterpret_cast<T*>(smraw);
    __shared__ __align__(8) uint64_t full[kStages];
    const int tid = threadIdx.x;
    const int64_t ntile = (n + TR - 1) / TR;
    const int64_t step = gridDim.x;

    auto issue = [&](int64_t tile, int st) {
        const int64_t row0 = tile * TR;
        const int rows = (int)((n - row0) < TR ? (n - row0) : TR);
        T* xs = sm + st * U::kSF;
        const uint32_t bytes = (uint32_t)rows * M * sizeof(T);
        mbar_expect_tx(&full[st], 2 * bytes);
        bulk_g2s(xs, X + row0 * M, bytes, &full[st]);
        bulk_g2s(xs + TR * M, Y + row0 * M, bytes, &full[st]);
    };

    if (tid == 0) {
        for (int s = 0; s < kStages; ++s) mbar_init(&full[s], 1);
        fence_barrier_init();
    }
    __syncthreads();
    int64_t issued = 0;
    for (int s = 0; s < kStages && blockIdx.x + s * step < ntile; ++s) {
        if (tid == 0) issue(blockIdx.x + s * step, s);
        ++issued;
    }
    // this thread's lane block (bi, bj) and row phase
    const bool active = tid < NB * PH;
    const int blk = tid % NB, ph = tid / NB;
    int bi = 0, bj = 0;
    {
        int k = 0;
        for (int cj = 0; cj < M / 8; ++cj)
            for (int ci = 0; ci < M / 4; ++ci)
                if (upper_block(ci, cj)) {
                    if (k == blk) {
                        bi = ci;
                        bj = cj;
                    }
                    ++k;
                }
    }
    typename Pol::R acc[4][8];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 8; ++b) Pol::zero(acc[a][b]);
    int64_t it = 0;
    for (int64_t tile = blockIdx.x; tile < ntile; tile += step, ++it) {
        const int st = (int)(it % kStages);
        const bool ok = mbar_wait(&full[st], (uint32_t)((it / kStages) & 1));
        if (__syncthreads_or(!ok)) {
            if (tid == 0) {
                atomicOr(err, 4);
                for (int64_t j = it; j < issued; ++j)
                    (void)mbar_wait(&full[j % kStages], (uint32_t)((j / kStages) & 1));
            }
            __syncthreads();
            return;
        }
        const T* xs = sm + st * U::kSF;
        const T* ys = xs + TR * M;
        const int64_t row0 = tile * TR;
        const int rows = (int)((n - row0) < TR ? (n - row0) : TR);
        if (active) {
            for (int r = ph; r < rows; r += PH) {
                T a[4], b[8];
                load4(xs + r * M + 4 * bi, a);
                load4(ys + r * M + 8 * bj, b);
                load4(ys + r * M + 8 * bj + 4, b + 4);
#pragma unroll
                for (int k = 0; k < 4; ++k)
#pragma unroll
                    for (int l = 0; l < 8; ++l) Pol::add(acc[k][l], a[k], b[l]);
            }
        }
        __syncthreads();   // every thread is done with this stage
        if (tid == 0) {
            const int64_t next = tile + kStages * step;
            if (next < ntile) issue(next, st);
        }
        if (tile + kStages * step < ntile) ++issued;
    }
    // every issued tile has been consumed: the staging memory is free for the reduction
    double* red = reinterpret_cast<double*>(smraw);      // [PH][NB][4 x 8]
    if (active) {
#pragma unroll
        for (int k = 0; k < 4; ++k)
#pragma unroll
            for (int l = 0; l < 8; ++l)
                red[(ph * NB + blk) * 32 + k * 8 + l] = Pol::out(acc[k][l]);
    }
    __syncthreads();
    double* out = partials + (int64_t)blockIdx.x * (kGramTile * kGramTile);
    for (int e = tid; e < M * M; e += kUThreads) {
        const int i = e / M, j = e - i * M;
        const int ci = i / 4, cj = j / 8;
        double s = 0.0;
        if (upper_block(ci, cj)) {
            int b = 0;
            for (int qj = 0; qj < M / 8; ++qj)
                for (int qi = 0; qi < M / 4; ++qi)
                    if (upper_block(qi, qj) && (qj < cj || (qj == cj && qi < ci))) ++b;
            for (int p = 0; p < PH; ++p) s += red[(p * NB + b) * 32 + (i % 4) * 8 + (j % 8)];
        }
        out[e] = s;
    }
}

// ---------------------------------------------------------------------------------------
// float64 CGS coefficient Gram C = X^T Y (X: P / Q window blocks of width Q, Y: one block of
// width Q): the whole P x Q output per CTA, an MP x MQ micro-tile per thread (P/MP x Q/MQ =
// 256 threads), every thread adding every row of the CTA's tiles in row order.  Row tiles
// (kGR rows of every block) are staged by bulk copies on the three-stage mbarrier pipeline,
// so loads overlap the FP64 work within the CTA.  Each CTA writes its P x Q partial
// (partials[cta*4096 + p*Q + q]) for k_gram_reduce.
// ---------------------------------------------------------------------------------------
constexpr int kGR = 32;

template <int P, int Q>
struct GramBulkShape {
    static_assert(P % Q == 0 && P <= 64 && Q <= 32, "bulk Gram shape");
    static constexpr int kSE = (P + Q) * kGR;                 // doubles per stage
    static constexpr size_t kSmem = (size_t)kStages * kSE * sizeof(double);
};

template <int P, int Q, int MP, int MQ>
__global__ void __launch_bounds__(kThreads)
k_gram_bulk_f64(MB<const double> X, MB<const double> Y, int64_t n, double* __restrict__ partials,
                int* err) {
    using S = GramBulkShape<P, Q>;
    constexpr int NB = P / Q, TQT = Q / MQ;
    static_assert((P / MP) * TQT == kThreads, "thread layout");
    extern __shared__ __align__(128) double gsm[];
    __shared__ __align__(8) uint64_t full[kStages];
    const int tid = threadIdx.x;
    const int64_t ntile = (n + kGR - 1) / kGR;
    const int64_t step = gridDim.x;

    auto issue = [&](int64_t tile, int st) {
        const int64_t row0 = tile * kGR;
        const int rows = (int)((n - row0) < kGR ? (n - row0) : kGR);
        double* xs = gsm + st * S::kSE;
        const uint32_t bytes = (uint32_t)rows * Q * sizeof(double);
        mbar_expect_tx(&full[st], bytes * (NB + 1));
#pragma unroll
        for (int b = 0; b < NB; ++b) bulk_g2s(xs + b * kGR * Q, X.blk(b) + row0 * Q, bytes, &full[st]);
        bulk_g2s(xs + NB * kGR * Q, Y.blk(0) + row0 * Q, bytes, &full[st]);
    };

    if (tid == 0) {
        for (int s = 0; s < kStages; ++s) mbar_init(&full[s], 1);
        fence_barrier_init();
    }
    __syncthreads();
    int64_t issued = 0;
    for (int s = 0; s < kStages && blockIdx.x + s * step < ntile; ++s) {
        if (tid == 0) issue(blockIdx.x + s * step, s);
        ++issued;
    }
    const int ti = tid / TQT, tj = tid % TQT;
    double acc[MP][MQ];
#pragma unroll
    for (int a = 0; a < MP; ++a)
#pragma unroll
        for (int b = 0; b < MQ; ++b) acc[a][b] = 0.0;
    int64_t it = 0;
    for (int64_t tile = blockIdx.x; tile < ntile; tile += step, ++it) {
        const int st = (int)(it % kStages);
        const bool ok = mbar_wait(&full[st], (uint32_t)((it / kStages) & 1));
        if (__syncthreads_or(!ok)) {
            if (tid == 0) {
                atomicOr(err, 4);
                for (int64_t j = it; j < issued; ++j)
                    (void)mbar_wait(&full[j % kStages], (uint32_t)((j / kStages) & 1));
            }
            __syncthreads();
            return;
        }
        const double* xs = gsm + st * S::kSE;
        const double* ys = xs + NB * kGR * Q;
        const int64_t row0 = tile * kGR;
        const int rows = (int)((n - row0) < kGR ? (n - row0) : kGR);
        for (int r = 0; r < rows; ++r) {
            double a[MP], b[MQ];
#pragma unroll
            for (int k = 0; k < MP; ++k) {
                const int pp = ti * MP + k;
                a[k] = xs[(pp / Q) * kGR * Q + r * Q + (pp % Q)];
            }
#pragma unroll
            for (int l = 0; l < MQ; ++l) b[l] = ys[r * Q + tj * MQ + l];
#pragma unroll
            for (int k = 0; k < MP; ++k)
#pragma unroll
                for (int l = 0; l < MQ; ++l) acc[k][l] = fma(a[k], b[l], acc[k][l]);
        }
        __syncthreads();   // every thread is done with this stage
        if (tid == 0) {
            const int64_t next = tile + kStages * step;
            if (next < ntile) issue(next, st);
        }
        if (tile + kStages * step < ntile) ++issued;
    }
    double* out = partials + (int64_t)blockIdx.x * (kGramTile * kGramTile);
#pragma unroll
    for (int k = 0; k < MP; ++k)
#pragma unroll
        for (int l = 0; l < MQ; ++l) out[(ti * MP + k) * Q + tj * MQ + l] = acc[k][l];
}

}  // namespace bulk
}  // namespace ekcg
