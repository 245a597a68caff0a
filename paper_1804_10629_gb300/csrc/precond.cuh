// Block Jacobi preconditioner application (Section 5): triangular solves with the IC(0)
// factor L of each diagonal block.
//
// The rows of every block are grouped into levels on the host: a row's level is one more
// than the highest level of the rows its equation reads (forward solve L y = x: the
// strictly lower entries of its row of L; backward solve L^T z = y: the entries below the
// diagonal in its column of L, stored row-wise as the strictly upper part of L^T).  One CTA
// per block walks its levels in order; the rows of a level (times the w columns of the
// block of vectors) are independent and spread over the CTA's threads, and a CTA barrier
// separates consecutive levels.  X is n x w row-major in the permuted row order and is
// overwritten in place (rows of a level read only rows of earlier levels).
#pragma once

#include <cstdint>

namespace ekcg {

// X <- L_d^{-1} X (forward arrays) or L_d^{-T} X (backward arrays) on the rows of every block.
// blk_lev[d] .. blk_lev[d+1]: the level indices of block d; lev_ptr[l] .. lev_ptr[l+1]: the
// positions in `rows` of level l; rp / ci / v: CSR (global permuted row and column indices)
// of the off-diagonal entries each row's equation reads; diag: the diagonal of L.
__global__ void __launch_bounds__(256)
k_bj_trsv(double* X, int w, const int32_t* __restrict__ blk_lev,
          const int32_t* __restrict__ lev_ptr, const int32_t* __restrict__ rows,
          const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
          const double* __restrict__ v, const double* __restrict__ diag) {
    const int d = blockIdx.x;
    for (int l = blk_lev[d]; l < blk_lev[d + 1]; ++l) {
        const int r0 = lev_ptr[l], r1 = lev_ptr[l + 1];
        const int cnt = (r1 - r0) * w;
        for (int e = threadIdx.x; e < cnt; e += blockDim.x) {
            const int i = rows[r0 + e / w];
            const int c = e - (e / w) * w;
            double s = X[(int64_t)i * w + c];
            for (int k = rp[i]; k < rp[i + 1]; ++k) s -= v[k] * X[(int64_t)ci[k] * w + c];
            X[(int64_t)i * w + c] = s / diag[i];
        }
        __syncthreads();
    }
}

}  // namespace ekcg
