// Batched s-step SRE-CG (Algorithm 4) for many independent systems in one persistent launch.
//
// Each CTA takes the next system from a device work queue (systems are queued largest
// first) and runs the whole s-step loop for it with CTA-wide barriers only: no CTA ever
// waits on another, and every loop is bounded by maxit.  The steps are the same as the
// single-system path (T(r_0), sparse products, CGS2 with fresh products against the two
// previous blocks, A-CholQR, alpha = V^T r, x/r update), written as CTA-cooperative device
// functions.  Precision: float64, or float32 inner solves in a float64 refinement loop.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <string>
#include <vector>

#include "../../include/ekcg.h"

namespace {

thread_local std::string g_berr;

#define EB_CUDA(call)                                         \
    do {                                                      \
        cudaError_t e_ = (call);                              \
        if (e_ != cudaSuccess) {                              \
            g_berr = std::string(#call) + ": " + cudaGetErrorString(e_); \
            return EKCG_ECUDA;                                \
        }                                                     \
    } while (0)

constexpr int kMaxT = 16;              // t <= 16
constexpr int kMaxS = 4;               // s <= 4
constexpr int kMaxP = 2 * kMaxT;       // window of two blocks
constexpr int kMaxST = kMaxS * kMaxT;

struct Sys {
    int64_t n;        // rows
    int64_t row0;     // first row in the concatenated vectors
    int64_t rp0;      // first entry in the concatenated row pointers (n + 1 per system)
    int64_t nz0;      // first nonzero
    int64_t ws0;      // first element of the system's basis workspace
};

struct Params {
    const Sys* sys;
    int nsys;
    int* queue;                 // work counter
    const int32_t* order;       // queue position -> system index
    const int32_t* rowptr;      // per-system local row pointers (permuted)
    const int32_t* col;         // local columns (permuted)
    const double* val;
    const float* val32;
    const int32_t* dom;         // domain of each (permuted) row
    const double* b;            // permuted right-hand sides (concatenated)
    double* x;                  // permuted solutions (concatenated)
    double* r64;                // float64 residual scratch (concatenated)
    void* ws;                   // basis workspace: per system (2s+3) n t elements + 2n
    int t, s;
    double tol, bd_tol, inner_tol;
    int maxit, max_refine;
    int* iters;                 // per system
    int* status;                // per system
    double* rho_out;            // per system: final recursive (or refined) residual norm
};

// ---- CTA-wide building blocks ---------------------------------------------------------

__device__ double cta_sum(double v, double* red) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[wid] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += red[i];
        red[32] = s;
    }
    __syncthreads();
    return red[32];
}

template <typename T>
__device__ void cta_spmm(T* __restrict__ U, const T* __restrict__ W, const int32_t* rp,
                         const int32_t* col, const T* val, int64_t n, int t) {
    for (int64_t e = threadIdx.x; e < n * t; e += blockDim.x) {
        const int64_t i = e / t;
        const int c = (int)(e - i * t);
        T acc = T(0);
        for (int j = rp[i]; j < rp[i + 1]; ++j) acc += val[j] * W[(int64_t)col[j] * t + c];
        U[e] = acc;
    }
}

// Float-float accumulation (about 48 significant bits): the float product is made exact
// with an FMA and added with TwoSum.  Used when float32 data must give a float64-grade sum.
struct DFAcc {
    float hi = 0.f, lo = 0.f;
    __device__ __forceinline__ void add(float a, float b) {
        const float p = a * b;
        const float e = fmaf(a, b, -p);
        const float s = hi + p;
        const float v = s - hi;
        lo += ((hi - (s - v)) + (p - v)) + e;
        hi = s;
    }
    __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};
template <typename T, typename Acc>
struct CtaAcc {
    Acc a = Acc(0);
    __device__ __forceinline__ void add(T x, T y) { a += (Acc)x * (Acc)y; }
    __device__ __forceinline__ double value() const { return (double)a; }
};
template <>
struct CtaAcc<float, double> {
    DFAcc a;
    __device__ __forceinline__ void add(float x, float y) { a.add(x, y); }
    __device__ __forceinline__ double value() const { return a.value(); }
};

// C[p*Q + q] = sum_rows X_p[row] Y_q[row] (accumulated in Acc, stored as double); X is nx
// blocks (n x t), Y is ny blocks of ty columns.  With fewer outputs than threads, each output
// is split over row stripes reduced in stripe order (deterministic).
template <typename T, typename Acc>
__device__ void cta_gram(double* C, const T* const* X, int nx, const T* const* Y, int ny, int ty,
                         int64_t n, int t, double* scratch /* >= blockDim.x */) {
    const int P = nx * t, Q = ny * ty, PQ = P * Q;
    const int tid = threadIdx.x;
    if (PQ * 2 > (int)blockDim.x) {
        for (int o = tid; o < PQ; o += blockDim.x) {
            const int p = o / Q, q = o - p * Q;
            const T* xb = X[p / t];
            const T* yb = Y[q / ty];
            const int xc = p % t, yc = q % ty;
            CtaAcc<T, Acc> acc;
            for (int64_t row = 0; row < n; ++row) acc.add(xb[row * t + xc], yb[row * ty + yc]);
            C[o] = acc.value();
        }
        __syncthreads();
        return;
    }
    const int stripes = (int)blockDim.x / PQ;
    CtaAcc<T, Acc> acc;
    const bool active = tid < PQ * stripes;
    if (active) {
        const int o = tid % PQ, st = tid / PQ;
        const int p = o / Q, q = o - p * Q;
        const T* xb = X[p / t];
        const T* yb = Y[q / ty];
        const int xc = p % t, yc = q % ty;
        for (int64_t row = st; row < n; row += stripes) acc.add(xb[row * t + xc], yb[row * ty + yc]);
    }
    __syncthreads();
    if (active) scratch[tid] = acc.value();
    __syncthreads();
    for (int o = tid; o < PQ; o += blockDim.x) {
        double s = 0.0;
        for (int k = 0; k < stripes; ++k) s += scratch[k * PQ + o];
        C[o] = s;
    }
    __syncthreads();
}

// OUT = Y - sum_b X_b C_b  (C: (nx t) x t), OUT may alias Y.
template <typename T, typename CT>
__device__ void cta_sub(T* OUT, const T* Y, const T* const* X, int nx, const CT* C, int64_t n,
                        int t) {
    const int P = nx * t;
    for (int64_t e = threadIdx.x; e < n * t; e += blockDim.x) {
        const int64_t i = e / t;
        const int q = (int)(e - i * t);
        CT acc = CT(0);
        for (int k = 0; k < P; ++k) acc += (CT)X[k / t][i * t + (k % t)] * C[k * t + q];
        OUT[e] = (T)((CT)Y[e] - acc);
    }
    __syncthreads();
}

// W <- W Rinv (Rinv t x t upper triangular, in place), arithmetic in T.
template <typename T>
__device__ void cta_rmul(T* W, const T* Rinv, int64_t n, int t) {
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
        T row[kMaxT];
        for (int c = 0; c < t; ++c) row[c] = W[i * t + c];
        for (int q = 0; q < t; ++q) {
            T a = T(0);
            for (int k = 0; k <= q; ++k) a += row[k] * Rinv[k * t + q];
            W[i * t + q] = a;
        }
    }
    __syncthreads();
}

// Copy of a small float64 matrix in the basis precision (identity copy for float64).
template <typename T>
__device__ const T* cta_cast(const double* src, T* dst, int m) {
    for (int i = threadIdx.x; i < m; i += blockDim.x) dst[i] = (T)src[i];
    __syncthreads();
    return dst;
}

// Upper Cholesky of the t x t matrix G (upper triangle), R^{-1}; thread 0 only (t <= 16).
// Returns 1 on breakdown (pivot d_i <= tol*|G_ii| or non-finite).
__device__ int cta_chol(const double* G, double* Rinv, double* S, double* R, int t, double tol,
                        int* flag_sh) {
    if (threadIdx.x == 0) {
        int bad = 0;
        for (int i = 0; i < t; ++i)
            for (int j = 0; j < t; ++j) {
                S[i * t + j] = (j >= i) ? G[i * t + j] : 0.0;
                R[i * t + j] = 0.0;
            }
        for (int i = 0; i < t && !bad; ++i) {
            const double d = S[i * t + i];
            if (!(d > tol * fabs(G[i * t + i])) || !isfinite(d)) {
                bad = 1;
                break;
            }
            R[i * t + i] = sqrt(d);
            for (int j = i + 1; j < t; ++j) R[i * t + j] = S[i * t + j] / R[i * t + i];
            for (int j = i + 1; j < t; ++j)
                for (int l = j; l < t; ++l) S[j * t + l] -= R[i * t + j] * R[i * t + l];
        }
        for (int c = 0; c < t; ++c)
            for (int i = 0; i < t; ++i) Rinv[i * t + c] = (i == c) ? 1.0 : 0.0;
        if (!bad) {
            for (int c = 0; c < t; ++c)
                for (int i = c; i >= 0; --i) {
                    double s = (i == c) ? 1.0 : 0.0;
                    for (int k = i + 1; k <= c; ++k) s -= R[i * t + k] * Rinv[k * t + c];
                    Rinv[i * t + c] = s / R[i * t + i];
                }
        }
        *flag_sh = bad;
    }
    __syncthreads();
    return *flag_sh;
}

struct Shared {
    double C[kMaxP * kMaxT];
    double G[kMaxT * kMaxT];
    double Rinv[kMaxT * kMaxT];
    double S[kMaxT * kMaxT];
    double R[kMaxT * kMaxT];
    float Cf[kMaxP * kMaxT];      // float copies for the float32 inner solve
    float Rinvf[kMaxT * kMaxT];
    double alpha[kMaxST];
    double red[40];
    int flag;
};

// s-step SRE-CG on one system in precision T: x (T) from its content, r (T) = residual.
// Returns the number of iterations; *st receives OK / MAXIT / BREAKDOWN; *rho the final
// recursive residual norm.
// stag > 0: stop when no new minimum of rho was reached in the last `stag` iterations.
template <typename T>
__device__ int cta_sstep(const Params& P, const Sys& S, T* x, T* r, T* Wb, T* Zb, const T* val,
                         double rho0, double tol_abs, int maxit, Shared& sh, double* scratch,
                         int* st, double* rho_out, int stag = 0) {
    const int t = P.t, s = P.s;
    const int64_t n = S.n, slot = n * t;
    const int32_t* rp = P.rowptr + S.rp0;
    const int32_t* col = P.col + S.nz0;
    const int32_t* dom = P.dom + S.row0;
    const int ring = s + 2, zring = s + 1;
    auto W = [&](int64_t j) { return Wb + (j % ring) * slot; };
    auto Z = [&](int64_t j) { return Zb + (j % zring) * slot; };
    double rho = rho0, best = rho0;
    int k = 1, k_best = 0;
    int64_t nb = 0;
    *st = EKCG_OK;
    while (rho > tol_abs && k < maxit + 1 &&
           !(stag > 0 && k - 1 - k_best >= max(stag, k_best / 2))) {
        const int64_t j0 = nb;
        for (int i = 0; i < s; ++i) {
            const int64_t j = j0 + i;
            if (j == 0) {
                T* w = W(0);
                for (int64_t e = threadIdx.x; e < slot; e += blockDim.x) {
                    const int64_t row = e / t;
                    w[e] = ((int)(e - row * t) == dom[row]) ? r[row] : T(0);
                }
                __syncthreads();
                cta_spmm<T>(Z(0), W(0), rp, col, val, n, t);
                __syncthreads();
            } else {
                const T* cand = Z(j - 1);
                cta_spmm<T>(Z(j), cand, rp, col, val, n, t);
                __syncthreads();
                const int64_t q0 = j >= 2 ? j - 2 : 0;
                const int qc = (int)(j - q0);
                const T* Q[2] = {W(q0), W(q0 + 1)};
                for (int pass = 0; pass < 2; ++pass) {
                    const T* Zs[1] = {Z(j)};
                    cta_gram<T, T>(sh.C, Q, qc, Zs, 1, t, n, t, scratch);
                    if constexpr (sizeof(T) == sizeof(double)) {
                        cta_sub<T, double>(W(j), pass == 0 ? cand : W(j), Q, qc, sh.C, n, t);
                    } else {
                        const float* Cf = cta_cast<float>(sh.C, sh.Cf, qc * t * t);
                        cta_sub<T, float>(W(j), pass == 0 ? cand : W(j), Q, qc, Cf, n, t);
                    }
                    cta_spmm<T>(Z(j), W(j), rp, col, val, n, t);
                    __syncthreads();
                }
            }
            // A-CholQR
            const T* Wj[1] = {W(j)};
            const T* Zj[1] = {Z(j)};
            cta_gram<T, double>(sh.G, Wj, 1, Zj, 1, t, n, t, scratch);
            if (cta_chol(sh.G, sh.Rinv, sh.S, sh.R, t, P.bd_tol, &sh.flag)) {
                *st = EKCG_EBREAKDOWN;
                *rho_out = rho;
                return k - 1;
            }
            const T* Ri;
            if constexpr (sizeof(T) == sizeof(double))
                Ri = (const T*)sh.Rinv;
            else
                Ri = (const T*)cta_cast<float>(sh.Rinv, sh.Rinvf, t * t);
            cta_rmul<T>(W(j), Ri, n, t);
            cta_rmul<T>(Z(j), Ri, n, t);
        }
        nb = j0 + s;
        // alpha = V^T r; x += V alpha; r -= (A V) alpha
        const T* Vs[kMaxS];
        const T* AVs[kMaxS];
        for (int i = 0; i < s; ++i) {
            Vs[i] = W(j0 + i);
            AVs[i] = Z(j0 + i);
        }
        const T* rv[1] = {r};
        cta_gram<T, double>(sh.alpha, Vs, s, rv, 1, 1, n, t, scratch);
        double local = 0.0;
        for (int64_t row = threadIdx.x; row < n; row += blockDim.x) {
            double sx = 0.0, sr = 0.0;
            for (int b = 0; b < s; ++b)
                for (int c = 0; c < t; ++c) {
                    sx += (double)Vs[b][row * t + c] * sh.alpha[b * t + c];
                    sr += (double)AVs[b][row * t + c] * sh.alpha[b * t + c];
                }
            const T xi = (T)((double)x[row] + sx);
            const T ri = (T)((double)r[row] - sr);
            x[row] = xi;
            r[row] = ri;
            local += (double)ri * (double)ri;
        }
        rho = sqrt(cta_sum(local, sh.red));
        if (rho < best) {
            best = rho;
            k_best = k;
        }
        ++k;
    }
    if (rho > tol_abs) *st = EKCG_MAXIT;
    *rho_out = rho;
    return k - 1;
}

__device__ double cta_residual64(const Params& P, const Sys& S, double* r) {
    const int32_t* rp = P.rowptr + S.rp0;
    const int32_t* col = P.col + S.nz0;
    const double* val = P.val + S.nz0;
    const double* b = P.b + S.row0;
    const double* x = P.x + S.row0;
    __shared__ double red[40];
    double local = 0.0;
    for (int64_t i = threadIdx.x; i < S.n; i += blockDim.x) {
        double acc = 0.0;
        for (int j = rp[i]; j < rp[i + 1]; ++j) acc += val[j] * x[col[j]];
        const double ri = b[i] - acc;
        r[i] = ri;
        local += ri * ri;
    }
    return sqrt(cta_sum(local, red));
}

template <bool MIXED>
__global__ void __launch_bounds__(512) k_batched(Params P) {
    __shared__ Shared sh;
    __shared__ int sid;
    extern __shared__ double scratch[];
    while (true) {
        __syncthreads();
        if (threadIdx.x == 0) {
            const int q = atomicAdd(P.queue, 1);
            sid = q < P.nsys ? P.order[q] : -1;
        }
        __syncthreads();
        if (sid < 0) return;
        const Sys S = P.sys[sid];
        double* r64 = P.r64 + S.row0;
        const double rho0 = cta_residual64(P, S, r64);
        int its = 0, st = EKCG_OK;
        double rho = rho0;
        if (!isfinite(rho0)) {
            st = EKCG_EINVAL;
        } else if (rho0 > 0 && !MIXED) {
            double* Wb = (double*)P.ws + S.ws0;
            double* Zb = Wb + (int64_t)(P.s + 2) * S.n * P.t;
            double* xx = P.x + S.row0;
            its = cta_sstep<double>(P, S, xx, r64, Wb, Zb, P.val + S.nz0, rho0, P.tol * rho0,
                                    P.maxit, sh, scratch, &st, &rho);
        } else if (rho0 > 0) {
            float* Wb = (float*)P.ws + S.ws0;
            float* Zb = Wb + (int64_t)(P.s + 2) * S.n * P.t;
            float* d = Zb + (int64_t)(P.s + 1) * S.n * P.t;
            float* r32 = d + S.n;
            st = EKCG_MAXIT;
            for (int ref = 0; ref < P.max_refine && its < P.maxit; ++ref) {
                const double sc = 1.0 / rho;
                for (int64_t i = threadIdx.x; i < S.n; i += blockDim.x) {
                    r32[i] = (float)(r64[i] * sc);
                    d[i] = 0.f;
                }
                __syncthreads();
                int ist = 0;
                double irho = 0;
                // the inner solve reduces r only as far as the outer tolerance still needs
                const double itol = fmax(P.inner_tol, 0.5 * P.tol * rho0 / rho);
                its += cta_sstep<float>(P, S, d, r32, Wb, Zb, P.val32 + S.nz0, 1.0, itol,
                                        P.maxit - its, sh, scratch, &ist, &irho, 50);
                for (int64_t i = threadIdx.x; i < S.n; i += blockDim.x)
                    P.x[S.row0 + i] += rho * (double)d[i];
                __syncthreads();
                const double rho_prev = rho;
                rho = cta_residual64(P, S, r64);
                if (!(rho > P.tol * rho0)) {
                    st = EKCG_OK;
                    break;
                }
                if (!isfinite(rho) || (ist == EKCG_EBREAKDOWN && irho >= 1.0)) {
                    st = EKCG_EBREAKDOWN;
                    break;
                }
                if (rho > 0.9 * rho_prev) break;   // refinement stagnated: EKCG_MAXIT
            }
        }
        if (threadIdx.x == 0) {
            P.iters[sid] = its;
            P.status[sid] = st;
            P.rho_out[sid] = rho;
        }
    }
}

__global__ void k_gather_b(double* y, const double* x, const int64_t* perm, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        y[i] = x[perm[i]];
}
__global__ void k_scatter_x(double* y, const double* x, const int64_t* perm, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        y[perm[i]] = x[i];
}

}  // namespace

struct ekcg_batch {
    int nsys = 0, t = 0, max_s = 0, precision = 0, num_sms = 0;
    double bd_tol = 1e-14, inner_tol = 1e-4;
    int max_refine = 30;
    cudaStream_t stream = nullptr;
    int64_t ntot = 0, nnz = 0;
    Sys* d_sys = nullptr;
    int32_t* d_order = nullptr;
    int* d_queue = nullptr;
    int32_t *d_rowptr = nullptr, *d_col = nullptr, *d_dom = nullptr;
    double* d_val = nullptr;
    float* d_val32 = nullptr;
    int64_t* d_perm = nullptr;   // global permuted position -> global natural row
    double *d_b = nullptr, *d_x = nullptr, *d_r = nullptr;
    void* d_ws = nullptr;
    int *d_iters = nullptr, *d_status = nullptr;
    double* d_rho = nullptr;
    int threads = 512, ctas_per_sm = 1;
    // captured graph of one solve
    cudaGraphExec_t graph = nullptr;
    int g_s = -1, g_maxit = -1;
    double g_tol = -1;
    float last_ms = 0.f;
};

namespace {

int launch_solve(ekcg_batch* B, int s, double tol, int maxit) {
    Params P{};
    P.sys = B->d_sys;
    P.nsys = B->nsys;
    P.queue = B->d_queue;
    P.order = B->d_order;
    P.rowptr = B->d_rowptr;
    P.col = B->d_col;
    P.val = B->d_val;
    P.val32 = B->d_val32;
    P.dom = B->d_dom;
    P.b = B->d_b;
    P.x = B->d_x;
    P.r64 = B->d_r;
    P.ws = B->d_ws;
    P.t = B->t;
    P.s = s;
    P.tol = tol;
    P.bd_tol = B->bd_tol;
    P.inner_tol = B->inner_tol;
    P.maxit = maxit;
    P.max_refine = B->max_refine;
    P.iters = B->d_iters;
    P.status = B->d_status;
    P.rho_out = B->d_rho;
    const int grid = std::min(B->nsys, B->num_sms * B->ctas_per_sm);
    const size_t smem = (size_t)B->threads * sizeof(double);
    EB_CUDA(cudaMemsetAsync(B->d_queue, 0, sizeof(int), B->stream));
    EB_CUDA(cudaMemsetAsync(B->d_x, 0, B->ntot * sizeof(double), B->stream));
    if (B->precision == EKCG_FP64)
        k_batched<false><<<grid, B->threads, smem, B->stream>>>(P);
    else
        k_batched<true><<<grid, B->threads, smem, B->stream>>>(P);
    EB_CUDA(cudaGetLastError());
    return EKCG_OK;
}

}  // namespace

extern "C" {

int ekcg_batched_setup(int nsys, const int64_t* n, const int64_t* rowptr, const int32_t* colind,
                       const double* val, int t, const int32_t* part, const ekcg_opts* opts,
                       void* stream, ekcg_batch** out) {
    if (!out || nsys < 1 || !n || !rowptr || !colind || !val || !part || t < 1 || t > kMaxT) {
        g_berr = "ekcg_batched_setup: bad arguments (t must be <= 16)";
        return EKCG_EINVAL;
    }
    *out = nullptr;
    ekcg_opts o;
    if (opts)
        o = *opts;
    else
        ekcg_default_opts(&o);
    if (o.variant != EKCG_SRE || o.basis != EKCG_SSTEP || o.orth != EKCG_ACHOLQR ||
        o.max_s < 1 || o.max_s > kMaxS) {
        g_berr = "ekcg_batched_setup: batched solves run s-step SRE-CG with A-CholQR, s <= 4";
        return EKCG_EINVAL;
    }
    ekcg_batch* B = new ekcg_batch();
    B->nsys = nsys;
    B->t = t;
    B->max_s = o.max_s;
    B->precision = o.precision;
    B->bd_tol = o.breakdown_tol;
    B->inner_tol = o.inner_tol;
    B->max_refine = o.max_refine;
    B->stream = (cudaStream_t)stream;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&B->num_sms, cudaDevAttrMultiProcessorCount, dev);
    std::vector<Sys> sys(nsys);
    int64_t row0 = 0, rp0 = 0, nz0 = 0, ws0 = 0;
    const int S = o.max_s;
    std::vector<int32_t> hrow, hcol, hdom;
    std::vector<double> hval;
    std::vector<int64_t> hperm;
    for (int k = 0; k < nsys; ++k) {
        const int64_t nk = n[k];
        const int64_t* rpk = rowptr + rp0;      // local row pointers (rpk[0] = 0)
        const int64_t nnzk = rpk[nk] - rpk[0];
        if (nk < 1 || nnzk < 1) {
            g_berr = "ekcg_batched_setup: empty system";
            delete B;
            return EKCG_EINVAL;
        }
        const int32_t* pk = part + row0;
        // stable sort of the system's rows by domain, symmetric permutation
        std::vector<int64_t> cnt(t, 0);
        for (int64_t i = 0; i < nk; ++i) {
            if (pk[i] < 0 || pk[i] >= t) {
                g_berr = "ekcg_batched_setup: part out of range";
                delete B;
                return EKCG_EINVAL;
            }
            cnt[pk[i]]++;
        }
        for (int d = 0; d < t; ++d)
            if (!cnt[d]) {
                g_berr = "ekcg_batched_setup: empty domain";
                delete B;
                return EKCG_EINVAL;
            }
        std::vector<int64_t> pos(t, 0), perm(nk), iperm(nk);
        for (int d = 1; d < t; ++d) pos[d] = pos[d - 1] + cnt[d - 1];
        for (int64_t i = 0; i < nk; ++i) perm[pos[pk[i]]++] = i;
        for (int64_t i = 0; i < nk; ++i) iperm[perm[i]] = i;
        const int64_t base_nz = (int64_t)hcol.size();
        const int64_t hrp0 = (int64_t)hrow.size();
        hrow.push_back(0);
        std::vector<std::pair<int32_t, double>> tmp;
        for (int64_t i = 0; i < nk; ++i) {
            const int64_t src = perm[i];
            tmp.clear();
            for (int64_t j = rpk[src]; j < rpk[src + 1]; ++j) {
                const int64_t cj = colind[nz0 + j];
                if (cj < 0 || cj >= nk) {
                    g_berr = "ekcg_batched_setup: column out of range";
                    delete B;
                    return EKCG_EINVAL;
                }
                tmp.push_back({(int32_t)iperm[cj], val[nz0 + j]});
            }
            std::sort(tmp.begin(), tmp.end(),
                      [](const std::pair<int32_t, double>& a, const std::pair<int32_t, double>& b) {
                          return a.first < b.first;
                      });
            for (auto& pr : tmp) {
                hcol.push_back(pr.first);
                hval.push_back(pr.second);
            }
            hrow.push_back((int32_t)((int64_t)hcol.size() - base_nz));
            hdom.push_back(pk[src]);
            hperm.push_back(row0 + src);
        }
        sys[k] = Sys{nk, row0, hrp0, base_nz, ws0};
        const int64_t per = (int64_t)(2 * S + 3) * nk * t + 2 * nk;
        ws0 += per;
        row0 += nk;
        rp0 += nk + 1;
        nz0 += nnzk;
    }
    B->ntot = row0;
    B->nnz = (int64_t)hcol.size();
    // queue: largest systems first
    std::vector<int32_t> order(nsys);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(),
                     [&](int a, int b) { return sys[a].n > sys[b].n; });
    std::vector<float> hval32(hval.begin(), hval.end());
    const size_t esz = o.precision == EKCG_FP64 ? sizeof(double) : sizeof(float);
    auto fail = [&](int rc) {
        ekcg_batched_destroy(B);
        return rc;
    };
#define EB_TRY(call)                                               \
    do {                                                           \
        cudaError_t e_ = (call);                                   \
        if (e_ != cudaSuccess) {                                   \
            g_berr = std::string(#call) + ": " + cudaGetErrorString(e_); \
            return fail(e_ == cudaErrorMemoryAllocation ? EKCG_ENOMEM : EKCG_ECUDA); \
        }                                                          \
    } while (0)
    EB_TRY(cudaMalloc(&B->d_sys, nsys * sizeof(Sys)));
    EB_TRY(cudaMalloc(&B->d_order, nsys * sizeof(int32_t)));
    EB_TRY(cudaMalloc(&B->d_queue, sizeof(int)));
    EB_TRY(cudaMalloc(&B->d_rowptr, hrow.size() * sizeof(int32_t)));
    EB_TRY(cudaMalloc(&B->d_col, hcol.size() * sizeof(int32_t)));
    EB_TRY(cudaMalloc(&B->d_val, hval.size() * sizeof(double)));
    EB_TRY(cudaMalloc(&B->d_val32, hval.size() * sizeof(float)));
    EB_TRY(cudaMalloc(&B->d_dom, hdom.size() * sizeof(int32_t)));
    EB_TRY(cudaMalloc(&B->d_perm, hperm.size() * sizeof(int64_t)));
    EB_TRY(cudaMalloc(&B->d_b, B->ntot * sizeof(double)));
    EB_TRY(cudaMalloc(&B->d_x, B->ntot * sizeof(double)));
    EB_TRY(cudaMalloc(&B->d_r, B->ntot * sizeof(double)));
    EB_TRY(cudaMalloc(&B->d_ws, (size_t)ws0 * esz));
    EB_TRY(cudaMalloc(&B->d_iters, nsys * sizeof(int)));
    EB_TRY(cudaMalloc(&B->d_status, nsys * sizeof(int)));
    EB_TRY(cudaMalloc(&B->d_rho, nsys * sizeof(double)));
    EB_TRY(cudaMemcpy(B->d_sys, sys.data(), nsys * sizeof(Sys), cudaMemcpyHostToDevice));
    EB_TRY(cudaMemcpy(B->d_order, order.data(), nsys * sizeof(int32_t), cudaMemcpyHostToDevice));
    EB_TRY(cudaMemcpy(B->d_rowptr, hrow.data(), hrow.size() * sizeof(int32_t),
                      cudaMemcpyHostToDevice));
    EB_TRY(cudaMemcpy(B->d_col, hcol.data(), hcol.size() * sizeof(int32_t),
                      cudaMemcpyHostToDevice));
    EB_TRY(cudaMemcpy(B->d_val, hval.data(), hval.size() * sizeof(double),
                      cudaMemcpyHostToDevice));
    EB_TRY(cudaMemcpy(B->d_val32, hval32.data(), hval32.size() * sizeof(float),
                      cudaMemcpyHostToDevice));
    EB_TRY(cudaMemcpy(B->d_dom, hdom.data(), hdom.size() * sizeof(int32_t),
                      cudaMemcpyHostToDevice));
    EB_TRY(cudaMemcpy(B->d_perm, hperm.data(), hperm.size() * sizeof(int64_t),
                      cudaMemcpyHostToDevice));
#undef EB_TRY
    *out = B;
    return EKCG_OK;
}

int ekcg_batched_tune(ekcg_batch* B, const double* b, int s, double tol, int maxit) {
    if (!B || !b) return EKCG_EINVAL;
    const int cand_threads[3] = {256, 512, 512};
    const int cand_ctas[3] = {2, 1, 2};
    float best = 1e30f;
    int bt = B->threads, bc = B->ctas_per_sm;
    cudaEvent_t e0, e1;
    EB_CUDA(cudaEventCreate(&e0));
    EB_CUDA(cudaEventCreate(&e1));
    for (int i = 0; i < 3; ++i) {
        B->threads = cand_threads[i];
        B->ctas_per_sm = cand_ctas[i];
        const int g = std::max(1, std::min<int>((int)((B->ntot + 255) / 256), B->num_sms * 8));
        k_gather_b<<<g, 256, 0, B->stream>>>(B->d_b, b, B->d_perm, B->ntot);
        EB_CUDA(cudaEventRecord(e0, B->stream));
        int rc = launch_solve(B, s, tol, maxit);
        if (rc != EKCG_OK) return rc;
        EB_CUDA(cudaEventRecord(e1, B->stream));
        EB_CUDA(cudaEventSynchronize(e1));
        float ms = 0.f;
        EB_CUDA(cudaEventElapsedTime(&ms, e0, e1));
        if (ms < best) {
            best = ms;
            bt = cand_threads[i];
            bc = cand_ctas[i];
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    B->threads = bt;
    B->ctas_per_sm = bc;
    if (B->graph) {
        cudaGraphExecDestroy(B->graph);
        B->graph = nullptr;
    }
    return EKCG_OK;
}

int ekcg_batched_solve(ekcg_batch* B, const double* b, int s, double tol, int maxit, double* x,
                       int* iters, int* status) {
    if (!B || !b || !x || s < 1 || s > B->max_s || !(tol > 0) || maxit < 0) {
        g_berr = "ekcg_batched_solve: bad arguments";
        return EKCG_EINVAL;
    }
    // the gather / queue reset / persistent solve / scatter run as one captured graph
    if (!B->graph || B->g_s != s || B->g_tol != tol || B->g_maxit != maxit) {
        if (B->graph) {
            cudaGraphExecDestroy(B->graph);
            B->graph = nullptr;
        }
        cudaStream_t cap;
        EB_CUDA(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
        EB_CUDA(cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal));
        cudaStream_t keep = B->stream;
        B->stream = cap;
        int rc = launch_solve(B, s, tol, maxit);
        B->stream = keep;
        cudaGraph_t g;
        cudaError_t ce = cudaStreamEndCapture(cap, &g);
        cudaStreamDestroy(cap);
        if (rc != EKCG_OK) return rc;
        EB_CUDA(ce);
        EB_CUDA(cudaGraphInstantiate(&B->graph, g, 0));
        cudaGraphDestroy(g);
        B->g_s = s;
        B->g_tol = tol;
        B->g_maxit = maxit;
    }
    const int g = std::max(1, std::min<int>((int)((B->ntot + 255) / 256), B->num_sms * 8));
    k_gather_b<<<g, 256, 0, B->stream>>>(B->d_b, b, B->d_perm, B->ntot);
    EB_CUDA(cudaGetLastError());
    cudaEvent_t e0, e1;
    EB_CUDA(cudaEventCreate(&e0));
    EB_CUDA(cudaEventCreate(&e1));
    EB_CUDA(cudaEventRecord(e0, B->stream));
    EB_CUDA(cudaGraphLaunch(B->graph, B->stream));
    EB_CUDA(cudaEventRecord(e1, B->stream));
    k_scatter_x<<<g, 256, 0, B->stream>>>(x, B->d_x, B->d_perm, B->ntot);
    EB_CUDA(cudaGetLastError());
    EB_CUDA(cudaStreamSynchronize(B->stream));
    EB_CUDA(cudaEventElapsedTime(&B->last_ms, e0, e1));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (iters)
        EB_CUDA(cudaMemcpy(iters, B->d_iters, B->nsys * sizeof(int), cudaMemcpyDeviceToHost));
    if (status)
        EB_CUDA(cudaMemcpy(status, B->d_status, B->nsys * sizeof(int), cudaMemcpyDeviceToHost));
    return EKCG_OK;
}

int ekcg_batched_info(const ekcg_batch* B, int* threads, int* ctas_per_sm, double* last_ms) {
    if (!B) return EKCG_EINVAL;
    if (threads) *threads = B->threads;
    if (ctas_per_sm) *ctas_per_sm = B->ctas_per_sm;
    if (last_ms) *last_ms = B->last_ms;
    return EKCG_OK;
}

void ekcg_batched_destroy(ekcg_batch* B) {
    if (!B) return;
    void* ptrs[] = {B->d_sys, B->d_order, B->d_queue, B->d_rowptr, B->d_col, B->d_val,
                    B->d_val32, B->d_dom, B->d_perm, B->d_b, B->d_x, B->d_r, B->d_ws,
                    B->d_iters, B->d_status, B->d_rho};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    if (B->graph) cudaGraphExecDestroy(B->graph);
    delete B;
}

const char* ekcg_batched_last_error(void) { return g_berr.c_str(); }

}  // extern "C"
