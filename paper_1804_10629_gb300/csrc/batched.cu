// Batched s-step SRE-CG (Algorithm 4) for many independent systems in one persistent launch.
//
// A group of CTAs -- one CTA, or the CTAs of one thread-block cluster -- takes the next
// system from a device work queue (systems are queued largest first) and runs the whole
// s-step loop for it.  Each CTA of the group owns a contiguous range of the system's rows;
// block inner products are reduced across the cluster through distributed shared memory,
// summed in rank order by every CTA, so that all CTAs hold bit-identical Gram matrices,
// Cholesky factors and residual norms and take the same branches.  Groups never wait on
// one another, and every loop is bounded by maxit.  The steps are the same as the
// single-system path (T(r_0), sparse products, CGS2 with fresh products against the two
// previous blocks, A-CholQR, alpha = V^T r, x/r update).  Precision: float64, or float32
// inner solves in a float64 refinement loop.
#include <cooperative_groups.h>
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
constexpr int kPart = kMaxP * kMaxT;   // largest reduced array (>= kMaxST)
constexpr int kMaxCluster = 8;         // portable cluster size
constexpr int kDefaultCluster = 4;     // CTAs per system unless set or tuned otherwise

namespace cg = cooperative_groups;

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
    int* switched;              // per system: 1 if the mixed solve continued in float64
};

// ---- group-wide building blocks -------------------------------------------------------

// The CTAs that solve one system: a single CTA (CL = false; barriers are __syncthreads) or
// the CTAs of one thread-block cluster (CL = true; barriers are cluster barriers, whose
// release/acquire semantics also order one CTA's global-memory writes before another CTA's
// reads).  CTA `rank` owns rows [lo, hi) of the system.
template <bool CL>
struct Grp {
    int rank = 0, size = 1;
    int64_t lo = 0, hi = 0;
    double* part = nullptr;   // 2 x kPart doubles of shared memory: this CTA's partial sums
    int flip = 0;
    __device__ void rows(int64_t n) {
        lo = n * rank / size;
        hi = n * (rank + 1) / size;
    }
    __device__ void sync() {
        if constexpr (CL)
            cg::this_cluster().sync();
        else
            __syncthreads();
    }
    // this CTA's partial-sum buffer for the next reduction
    __device__ double* buf() { return part + flip * kPart; }
    // out[i] = sum over the group's CTAs, in rank order, of their buf()[i] (i < m); every CTA
    // forms the same sums.  The two buffers alternate, so one barrier per reduction is
    // enough: a CTA writes a buffer again only after passing the next reduction's barrier,
    // which every CTA reaches after reading the buffer.
    __device__ void reduce(double* out, int m) {
        if constexpr (CL) {
            sync();
            cg::cluster_group cl = cg::this_cluster();
            double* mine = buf();
            for (int i = threadIdx.x; i < m; i += blockDim.x) {
                double s = 0.0;
                for (int c = 0; c < size; ++c) s += cl.map_shared_rank(mine, c)[i];
                out[i] = s;
            }
            flip ^= 1;
            __syncthreads();
        }
    }
};

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

// Sum of v over the group (red: >= 34 doubles of shared memory).
template <bool CL>
__device__ double grp_sum(Grp<CL>& g, double v, double* red) {
    const double local = cta_sum(v, red);
    if constexpr (!CL) {
        return local;
    } else {
        if (threadIdx.x == 0) g.buf()[0] = local;
        g.reduce(red + 33, 1);
        return red[33];
    }
}

// Load of a vector entry that another CTA of the cluster may have written in this launch:
// taken from L2 (ld.global.cg), so it never depends on a line cached in this SM's L1.
template <bool CL, typename T>
__device__ __forceinline__ T ld_group(const T* p) {
    if constexpr (CL)
        return __ldcg(p);
    else
        return *p;
}

// U = A W on this CTA's rows (W is read at any row of the system).
template <typename T, bool CL>
__device__ void grp_spmm(const Grp<CL>& g, T* U, const T* W, const int32_t* __restrict__ rp,
                         const int32_t* __restrict__ col, const T* __restrict__ val, int t) {
    for (int64_t e = g.lo * t + threadIdx.x; e < g.hi * t; e += blockDim.x) {
        const int64_t i = e / t;
        const int c = (int)(e - i * t);
        T acc = T(0);
        for (int j = rp[i]; j < rp[i + 1]; ++j)
            acc += val[j] * ld_group<CL>(W + (int64_t)col[j] * t + c);
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

// C[p*Q + q] = sum over the system's rows of X_p[row] Y_q[row] (accumulated in Acc, stored as
// double); X is nx blocks (n x t), Y is ny blocks of ty columns.  Each CTA sums its own rows;
// with fewer outputs than threads, each output is split over row stripes reduced in stripe
// order; the group's partials are then reduced in rank order (deterministic).
template <typename T, typename Acc, bool CL>
__device__ void grp_gram(Grp<CL>& g, double* C, const T* const* X, int nx, const T* const* Y,
                         int ny, int ty, int t, double* scratch /* >= blockDim.x */) {
    const int P = nx * t, Q = ny * ty, PQ = P * Q;
    const int tid = threadIdx.x;
    const int64_t lo = g.lo, hi = g.hi;
    double* dst = CL ? g.buf() : C;
    if (PQ * 2 > (int)blockDim.x) {
        for (int o = tid; o < PQ; o += blockDim.x) {
            const int p = o / Q, q = o - p * Q;
            const T* xb = X[p / t];
            const T* yb = Y[q / ty];
            const int xc = p % t, yc = q % ty;
            CtaAcc<T, Acc> acc;
            for (int64_t row = lo; row < hi; ++row) acc.add(xb[row * t + xc], yb[row * ty + yc]);
            dst[o] = acc.value();
        }
        __syncthreads();
    } else {
        const int stripes = (int)blockDim.x / PQ;
        CtaAcc<T, Acc> acc;
        const bool active = tid < PQ * stripes;
        if (active) {
            const int o = tid % PQ, st = tid / PQ;
            const int p = o / Q, q = o - p * Q;
            const T* xb = X[p / t];
            const T* yb = Y[q / ty];
            const int xc = p % t, yc = q % ty;
            for (int64_t row = lo + st; row < hi; row += stripes)
                acc.add(xb[row * t + xc], yb[row * ty + yc]);
        }
        __syncthreads();
        if (active) scratch[tid] = acc.value();
        __syncthreads();
        for (int o = tid; o < PQ; o += blockDim.x) {
            double s = 0.0;
            for (int k = 0; k < stripes; ++k) s += scratch[k * PQ + o];
            dst[o] = s;
        }
        __syncthreads();
    }
    g.reduce(C, PQ);
}

// OUT = Y - sum_b X_b C_b on this CTA's rows (C: (nx t) x t); OUT may alias Y.
template <typename T, typename CT, bool CL>
__device__ void grp_sub(const Grp<CL>& g, T* OUT, const T* Y, const T* const* X, int nx,
                        const CT* C, int t) {
    const int P = nx * t;
    for (int64_t e = g.lo * t + threadIdx.x; e < g.hi * t; e += blockDim.x) {
        const int64_t i = e / t;
        const int q = (int)(e - i * t);
        CT acc = CT(0);
        for (int k = 0; k < P; ++k) acc += (CT)X[k / t][i * t + (k % t)] * C[k * t + q];
        OUT[e] = (T)((CT)Y[e] - acc);
    }
    __syncthreads();
}

// W <- W Rinv on this CTA's rows (Rinv t x t upper triangular, in place), arithmetic in T.
template <typename T, bool CL>
__device__ void grp_rmul(const Grp<CL>& g, T* W, const T* Rinv, int t) {
    for (int64_t i = g.lo + threadIdx.x; i < g.hi; i += blockDim.x) {
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
// Every CTA of a group factors the same G (bit-identical after the rank-order reduction).
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
    double part[2 * kPart];       // cluster partial sums (two alternating buffers)
    int flag;
};

// s-step SRE-CG on one system in precision T: x (T) from its content, r (T) = residual.
// Returns the number of iterations; *st receives OK / MAXIT / BREAKDOWN; *rho the final
// recursive residual norm.  Every CTA of the group returns the same values.
// stag > 0: stop when no new minimum of rho was reached in the last `stag` iterations.
template <typename T, bool CL>
__device__ int cta_sstep(const Params& P, const Sys& S, Grp<CL>& g, T* x, T* r, T* Wb, T* Zb,
                         const T* val, double rho0, double tol_abs, int maxit, Shared& sh,
                         double* scratch, int* st, double* rho_out, int stag = 0) {
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
                for (int64_t e = g.lo * t + threadIdx.x; e < g.hi * t; e += blockDim.x) {
                    const int64_t row = e / t;
                    w[e] = ((int)(e - row * t) == dom[row]) ? r[row] : T(0);
                }
                g.sync();
                grp_spmm<T>(g, Z(0), W(0), rp, col, val, t);
                __syncthreads();
            } else {
                const T* cand = Z(j - 1);
                if constexpr (CL) g.sync();   // Z(j-1) complete on every CTA's rows
                grp_spmm<T>(g, Z(j), cand, rp, col, val, t);
                __syncthreads();
                const int64_t q0 = j >= 2 ? j - 2 : 0;
                const int qc = (int)(j - q0);
                const T* Q[2] = {W(q0), W(q0 + 1)};
                for (int pass = 0; pass < 2; ++pass) {
                    const T* Zs[1] = {Z(j)};
                    grp_gram<T, T>(g, sh.C, Q, qc, Zs, 1, t, t, scratch);
                    if constexpr (sizeof(T) == sizeof(double)) {
                        grp_sub<T, double>(g, W(j), pass == 0 ? cand : W(j), Q, qc, sh.C, t);
                    } else {
                        const float* Cf = cta_cast<float>(sh.C, sh.Cf, qc * t * t);
                        grp_sub<T, float>(g, W(j), pass == 0 ? cand : W(j), Q, qc, Cf, t);
                    }
                    if constexpr (CL) g.sync();   // W(j) complete on every CTA's rows
                    grp_spmm<T>(g, Z(j), W(j), rp, col, val, t);
                    __syncthreads();
                }
            }
            // A-CholQR
            const T* Wj[1] = {W(j)};
            const T* Zj[1] = {Z(j)};
            grp_gram<T, double>(g, sh.G, Wj, 1, Zj, 1, t, t, scratch);
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
            grp_rmul<T>(g, W(j), Ri, t);
            grp_rmul<T>(g, Z(j), Ri, t);
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
        grp_gram<T, double>(g, sh.alpha, Vs, s, rv, 1, 1, t, scratch);
        double local = 0.0;
        for (int64_t row = g.lo + threadIdx.x; row < g.hi; row += blockDim.x) {
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
        rho = sqrt(grp_sum(g, local, sh.red));
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

// r = b - A x (float64) on this CTA's rows; returns ||r|| over the system.  x is read at any
// row, so every CTA's x must be complete (a group barrier) before the call.
template <bool CL>
__device__ double cta_residual64(Grp<CL>& g, const Params& P, const Sys& S, double* r) {
    const int32_t* rp = P.rowptr + S.rp0;
    const int32_t* col = P.col + S.nz0;
    const double* val = P.val + S.nz0;
    const double* b = P.b + S.row0;
    const double* x = P.x + S.row0;
    __shared__ double red[40];
    double local = 0.0;
    for (int64_t i = g.lo + threadIdx.x; i < g.hi; i += blockDim.x) {
        double acc = 0.0;
        for (int j = rp[i]; j < rp[i + 1]; ++j) acc += val[j] * ld_group<CL>(x + col[j]);
        const double ri = b[i] - acc;
        r[i] = ri;
        local += ri * ri;
    }
    return sqrt(grp_sum(g, local, red));
}

template <bool MIXED, bool CL>
__global__ void __launch_bounds__(512) k_batched(Params P) {
    __shared__ Shared sh;
    __shared__ int sid_sh;
    extern __shared__ double scratch[];
    Grp<CL> g;
    g.part = sh.part;
    if constexpr (CL) {
        g.rank = (int)cg::this_cluster().block_rank();
        g.size = (int)cg::this_cluster().num_blocks();
    }
    while (true) {
        int sid;
        if constexpr (CL) {
            // rank 0 takes the next system; the others read its choice from its shared memory
            if (g.rank == 0 && threadIdx.x == 0) {
                const int q = atomicAdd(P.queue, 1);
                sid_sh = q < P.nsys ? P.order[q] : -1;
            }
            g.sync();
            sid = *cg::this_cluster().map_shared_rank(&sid_sh, 0);
            g.sync();   // read by every CTA before rank 0 exits or takes the next system
        } else {
            __syncthreads();
            if (threadIdx.x == 0) {
                const int q = atomicAdd(P.queue, 1);
                sid_sh = q < P.nsys ? P.order[q] : -1;
            }
            __syncthreads();
            sid = sid_sh;
        }
        if (sid < 0) return;
        const Sys S = P.sys[sid];
        g.rows(S.n);
        double* r64 = P.r64 + S.row0;
        const double rho0 = cta_residual64(g, P, S, r64);
        int its = 0, st = EKCG_OK;
        double rho = rho0;
        if (!isfinite(rho0)) {
            st = EKCG_EINVAL;
        } else if (rho0 > 0 && !MIXED) {
            double* Wb = (double*)P.ws + S.ws0;
            double* Zb = Wb + (int64_t)(P.s + 2) * S.n * P.t;
            double* xx = P.x + S.row0;
            its = cta_sstep<double>(P, S, g, xx, r64, Wb, Zb, P.val + S.nz0, rho0, P.tol * rho0,
                                    P.maxit, sh, scratch, &st, &rho);
        } else if (rho0 > 0) {
            // float32 basis inside the system's workspace (sized for float64: see below)
            float* Wb = reinterpret_cast<float*>((double*)P.ws + S.ws0);
            float* Zb = Wb + (int64_t)(P.s + 2) * S.n * P.t;
            float* d = Zb + (int64_t)(P.s + 1) * S.n * P.t;
            float* r32 = d + S.n;
            st = EKCG_MAXIT;
            bool to64 = false;
            for (int ref = 0; ref < P.max_refine && its < P.maxit; ++ref) {
                const double sc = 1.0 / rho;
                for (int64_t i = g.lo + threadIdx.x; i < g.hi; i += blockDim.x) {
                    r32[i] = (float)(r64[i] * sc);
                    d[i] = 0.f;
                }
                __syncthreads();
                int ist = 0;
                double irho = 0;
                // the inner solve reduces r only as far as the outer tolerance still needs
                const double itol = fmax(P.inner_tol, 0.5 * P.tol * rho0 / rho);
                its += cta_sstep<float>(P, S, g, d, r32, Wb, Zb, P.val32 + S.nz0, 1.0, itol,
                                        P.maxit - its, sh, scratch, &ist, &irho, 50);
                for (int64_t i = g.lo + threadIdx.x; i < g.hi; i += blockDim.x)
                    P.x[S.row0 + i] += rho * (double)d[i];
                g.sync();   // the residual reads x on every CTA's rows
                const double rho_prev = rho;
                rho = cta_residual64(g, P, S, r64);
                if (!(rho > P.tol * rho0)) {
                    st = EKCG_OK;
                    break;
                }
                if (!isfinite(rho) || (ist == EKCG_EBREAKDOWN && irho >= 1.0)) {
                    st = EKCG_EBREAKDOWN;
                    break;
                }
                if (rho > 0.9 * rho_prev) {   // refinement stagnated (kappa eps32 near 1)
                    to64 = true;
                    break;
                }
            }
            if (to64 && its < P.maxit) {
                // precision switch for this system only: continue in float64 from the refined
                // x and its float64 residual, in the same workspace (every CTA of the group
                // has finished with the float32 basis: the residual above ended in a group
                // barrier)
                double* Wd = (double*)P.ws + S.ws0;
                double* Zd = Wd + (int64_t)(P.s + 2) * S.n * P.t;
                int st64 = EKCG_OK;
                double rho64 = rho;
                its += cta_sstep<double>(P, S, g, P.x + S.row0, r64, Wd, Zd, P.val + S.nz0, rho,
                                         P.tol * rho0, P.maxit - its, sh, scratch, &st64, &rho64);
                st = st64;
                rho = rho64;
                if (g.rank == 0 && threadIdx.x == 0) P.switched[sid] = 1;
            }
        }
        if (g.rank == 0 && threadIdx.x == 0) {
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
    int *d_iters = nullptr, *d_status = nullptr, *d_switched = nullptr;
    double* d_rho = nullptr;
    int threads = 512, ctas_per_sm = 1;
    int cluster = 1;            // CTAs per system (a thread-block cluster when > 1)
    int groups = 0;             // persistent groups launched (CTAs / cluster)
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
    P.switched = B->d_switched;
    const size_t smem = (size_t)B->threads * sizeof(double);
    EB_CUDA(cudaMemsetAsync(B->d_queue, 0, sizeof(int), B->stream));
    EB_CUDA(cudaMemsetAsync(B->d_switched, 0, B->nsys * sizeof(int), B->stream));
    EB_CUDA(cudaMemsetAsync(B->d_x, 0, B->ntot * sizeof(double), B->stream));
    const bool mixed = B->precision != EKCG_FP64;
    if (B->cluster == 1) {
        const int grid = B->groups;
        if (!mixed)
            k_batched<false, false><<<grid, B->threads, smem, B->stream>>>(P);
        else
            k_batched<true, false><<<grid, B->threads, smem, B->stream>>>(P);
    } else {
        cudaLaunchConfig_t cfg = {};
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = (unsigned)B->cluster;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.gridDim = dim3((unsigned)(B->groups * B->cluster));
        cfg.blockDim = dim3((unsigned)B->threads);
        cfg.dynamicSmemBytes = smem;
        cfg.stream = B->stream;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        if (!mixed)
            EB_CUDA(cudaLaunchKernelEx(&cfg, k_batched<false, true>, P));
        else
            EB_CUDA(cudaLaunchKernelEx(&cfg, k_batched<true, true>, P));
    }
    EB_CUDA(cudaGetLastError());
    return EKCG_OK;
}

// Launch shape: `threads` per CTA, `cluster` CTAs per system, at most `ctas_per_sm` CTAs per
// SM.  The persistent grid holds as many groups as can be resident at once (never more than
// there are systems), so every group runs from the start; groups never wait on one another.
int set_shape(ekcg_batch* B, int threads, int ctas_per_sm, int cluster) {
    if ((threads != 256 && threads != 512) || ctas_per_sm < 1 || ctas_per_sm > 2 ||
        (cluster != 1 && cluster != 2 && cluster != 4 && cluster != kMaxCluster)) {
        g_berr = "ekcg_batched_set_shape: threads in {256, 512}, ctas_per_sm in {1, 2}, "
                 "cluster in {1, 2, 4, 8}";
        return EKCG_EINVAL;
    }
    const bool mixed = B->precision != EKCG_FP64;
    const size_t smem = (size_t)threads * sizeof(double);
    int groups = 0;
    if (cluster == 1) {
        int per_sm = 0;
        EB_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(
            &per_sm, mixed ? k_batched<true, false> : k_batched<false, false>, threads, smem));
        groups = B->num_sms * std::min(per_sm, ctas_per_sm);
    } else {
        cudaLaunchConfig_t cfg = {};
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = (unsigned)cluster;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.gridDim = dim3((unsigned)(cluster * B->num_sms));
        cfg.blockDim = dim3((unsigned)threads);
        cfg.dynamicSmemBytes = smem;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        int nc = 0;
        EB_CUDA(cudaOccupancyMaxActiveClusters(
            &nc, (const void*)(mixed ? k_batched<true, true> : k_batched<false, true>), &cfg));
        groups = std::min(nc, B->num_sms * ctas_per_sm / cluster);
    }
    if (groups < 1) {
        g_berr = "ekcg_batched_set_shape: no resident group of this shape";
        return EKCG_EINVAL;
    }
    B->threads = threads;
    B->ctas_per_sm = ctas_per_sm;
    B->cluster = cluster;
    B->groups = std::min(groups, B->nsys);
    if (B->graph) {
        cudaGraphExecDestroy(B->graph);
        B->graph = nullptr;
    }
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
    // float64-sized in both precisions: a mixed system whose float32 refinement stagnates
    // continues in float64 in the same workspace
    const size_t esz = sizeof(double);
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
    EB_TRY(cudaMalloc(&B->d_switched, nsys * sizeof(int)));
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
    const int rc = set_shape(B, 512, 1, kDefaultCluster);
    if (rc != EKCG_OK) return fail(rc);
    *out = B;
    return EKCG_OK;
}

int ekcg_batched_tune(ekcg_batch* B, const double* b, int s, double tol, int maxit) {
    if (!B || !b || s < 1 || s > B->max_s || !(tol > 0) || maxit < 0) return EKCG_EINVAL;
    constexpr int kCand = 7;
    const int cand_threads[kCand] = {512, 256, 512, 512, 512, 256, 256};
    const int cand_ctas[kCand] = {1, 2, 1, 1, 1, 2, 2};
    const int cand_cluster[kCand] = {1, 1, 2, 4, 8, 4, 8};
    float best = 1e30f;
    int bt = B->threads, bc = B->ctas_per_sm, bk = B->cluster;
    cudaEvent_t e0, e1;
    EB_CUDA(cudaEventCreate(&e0));
    EB_CUDA(cudaEventCreate(&e1));
    for (int i = 0; i < kCand; ++i) {
        if (set_shape(B, cand_threads[i], cand_ctas[i], cand_cluster[i]) != EKCG_OK) continue;
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
            bk = cand_cluster[i];
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return set_shape(B, bt, bc, bk);
}

int ekcg_batched_set_shape(ekcg_batch* B, int threads, int ctas_per_sm, int cluster) {
    if (!B) return EKCG_EINVAL;
    return set_shape(B, threads, ctas_per_sm, cluster);
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

int ekcg_batched_info(const ekcg_batch* B, int* threads, int* ctas_per_sm, int* cluster,
                      int* groups, double* last_ms) {
    if (!B) return EKCG_EINVAL;
    if (threads) *threads = B->threads;
    if (ctas_per_sm) *ctas_per_sm = B->ctas_per_sm;
    if (cluster) *cluster = B->cluster;
    if (groups) *groups = B->groups;
    if (last_ms) *last_ms = B->last_ms;
    return EKCG_OK;
}

int ekcg_batched_precision_switches(const ekcg_batch* B, int* count) {
    if (!B || !count) return EKCG_EINVAL;
    std::vector<int> h(B->nsys);
    EB_CUDA(cudaMemcpyAsync(h.data(), B->d_switched, B->nsys * sizeof(int),
                            cudaMemcpyDeviceToHost, B->stream));
    EB_CUDA(cudaStreamSynchronize(B->stream));
    *count = 0;
    for (int v : h) *count += v != 0;
    return EKCG_OK;
}

void ekcg_batched_destroy(ekcg_batch* B) {
    if (!B) return;
    void* ptrs[] = {B->d_sys, B->d_order, B->d_queue, B->d_rowptr, B->d_col, B->d_val,
                    B->d_val32, B->d_dom, B->d_perm, B->d_b, B->d_x, B->d_r, B->d_ws,
                    B->d_iters, B->d_status, B->d_rho, B->d_switched};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    if (B->graph) cudaGraphExecDestroy(B->graph);
    delete B;
}

const char* ekcg_batched_last_error(void) { return g_berr.c_str(); }

}  // extern "C"
