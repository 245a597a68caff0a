// Float64-accurate tall-skinny contractions on the bf16 tensor cores (tcgen05, sm_103a).
//
// The CGS update W <- W - Q C of the A-orthonormalisation (Section 3.1, Section 4) is a
// product of an n x P block by a small P x Q matrix.  GB300's float64 FMA pipe retires about
// two FMAs per SM cycle, so in float64 this product runs twenty times below the HBM
// roofline.  Here it runs as a split ("Ozaki") product on the bf16 tensor cores:
//
//   * each row i of X (P values) is scaled by its largest binade, 2^{e_i - 1022}, and its
//     magnitudes cut into a 63-bit fixed-point integer F = sum_a x_a 2^{63-7a}, nine 7-bit
//     slices x_a in [0, 127] carrying the sign of the value (exact in bf16);
//   * each column q of C is cut the same way against its own binade 2^{f_q - 1022};
//   * the slice products are integers below 2^14, so over K = P <= 64 terms and up to nine
//     slice pairs (a, b) with a + b = g the fp32 accumulator of tcgen05.mma holds the exact
//     group sum G_g = sum_{a+b=g} sum_k x_a[i,k] c_b[k,q] (|G_g| < 2^24);
//   * the 45 pairs with a + b <= 10 form nine groups g = 2..10, each in its own TMEM
//     accumulator (128 lanes = rows, Q columns); the dropped pairs and the truncation of F
//     weigh at most about 2^-60 of max|X_i| max|C_q| per term, below one float64 rounding of
//     every term within 2^7 of that product;
//   * the epilogue combines the nine exact groups in 64-bit integers,
//     V = sum_g G_g 2^{7(10-g)} (kept as V / 2^14 rounded to the nearest integer, below
//     2^62), converts it once to float64 and applies the scale and the subtraction with one
//     fused multiply-add: OUT = Y - (V / 2^14) 2^{e_i + f_q - 2100}.
//
// Tensor-core mechanics: A (X slices, 128 rows x K) and B (C slices, Q x K) sit in shared
// memory in the canonical K-major no-swizzle layout of 8 x 16-byte core matrices (leading
// byte offset = distance of core matrices along K, stride byte offset = along M / N); one
// thread issues kind::f16 MMAs (bf16 x bf16 -> fp32, M = 128, N = Q, K = 16) into the
// accumulators allocated in tensor memory, commits them to an mbarrier, and the epilogue
// warps read the accumulators back with tcgen05.ld (warp w reads lanes 32 (w % 4) .. +31).
// Every mbarrier wait is bounded: a wait that runs out sets bit 2 of *err; the CTA then
// waits (bounded) for its outstanding MMAs, frees its tensor memory and returns.
#pragma once

#include <cstdint>

#include "bulk.cuh"
#include "kernels.cuh"

namespace ekcg {
namespace oz {

constexpr int kThreads = 256;
constexpr int kTile = 128;      // rows of X per tile (M of one MMA)
constexpr int kSlices = 9;      // 7-bit slices of the 63-bit fixed-point magnitude
constexpr int kGroups = 9;      // slice-pair groups g = a + b = 2..10
constexpr int kMaxN = 256;      // largest N of one tcgen05.mma (M = 64 or 128)
constexpr int kKC = 32;         // columns of X sliced per stage (K per stage)

// ---- tcgen05 / descriptor helpers ------------------------------------------------------
// Shared-memory matrix descriptor, K-major, no swizzle: start address, leading byte offset
// (K direction), stride byte offset (M / N direction), descriptor version 1 (bits 46-47).
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}
// Instruction descriptor of kind::f16: fp32 accumulator (bits 4-5 = 1), A and B bf16 (bits
// 7-9, 10-12 = 1), both K-major, N >> 3 at bits 17-22, M >> 4 at bits 24-28.
__host__ __device__ constexpr uint32_t idesc_bf16_f32(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) |
           ((uint32_t)(M >> 4) << 24);
}
__device__ __forceinline__ void tmem_alloc(uint32_t* slot, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     bulk::smem_addr(slot)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr),
                 "r"(ncols)
                 : "memory");
}
__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
// generic-proxy shared-memory writes -> visible to the tensor core (async proxy)
__device__ __forceinline__ void fence_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc,
                                         uint32_t idesc, uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}
// arrive on the mbarrier once every MMA this thread issued before has completed
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            bulk::smem_addr(bar))
        : "memory");
}
// 32 lanes x 8 consecutive 32-bit columns: this thread's lane, columns taddr.col .. +7
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float (&v)[8]) {
    uint32_t r[8];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7])
        : "r"(taddr)
        : "memory");
#pragma unroll
    for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}
// 32 lanes x 4 consecutive 32-bit columns
__device__ __forceinline__ void tmem_ld4(uint32_t taddr, float (&v)[4]) {
    uint32_t r[4];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0, %1, %2, %3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(taddr)
                 : "memory");
#pragma unroll
    for (int i = 0; i < 4; ++i) v[i] = __uint_as_float(r[i]);
}
// 32 lanes x 2 consecutive 32-bit columns
__device__ __forceinline__ void tmem_ld2(uint32_t taddr, float (&v)[2]) {
    uint32_t r[2];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x2.b32 {%0, %1}, [%2];"
                 : "=r"(r[0]), "=r"(r[1])
                 : "r"(taddr)
                 : "memory");
    v[0] = __uint_as_float(r[0]);
    v[1] = __uint_as_float(r[1]);
}
__device__ __forceinline__ void tmem_wait_ld() {
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// the nine exact group sums G_2 .. G_10 combined into V / 2^14, V = sum_g G_g 2^{7(10-g)}
// (|G_g| < 2^24, |G_2| < 2^21): G_2 2^42 + G_3 2^35 + ... + G_8 + G_9 / 2^7 + G_10 / 2^14,
// the last two rounded to the nearest integer (unbiased: the rounding errors of the tiles do
// not add up in one direction), within one unit of V / 2^14, below 2^62.  The terms below
// 2^32 are added by 32 x 32 -> 64-bit multiply-adds, the two top terms into the high word.
__device__ __forceinline__ long long combine_groups(const float (&g)[kGroups]) {
    // each group converted where it is added: few registers live at a time
    long long acc = (long long)(__float2int_rn(g[1]) * 8 + __float2int_rn(g[0]) * 1024) << 32;
    acc += (long long)__float2int_rn(g[2]) * 268435456;
    acc += (long long)__float2int_rn(g[3]) * 2097152;
    acc += (long long)__float2int_rn(g[4]) * 16384;
    acc += (long long)__float2int_rn(g[5]) * 128;
    return acc + (__float2int_rn(g[6]) + ((__float2int_rn(g[7]) + 64) >> 7) +
                  ((__float2int_rn(g[8]) + 8192) >> 14));
}
// 2^{ex - 1023} for a biased exponent ex: 0 below the normal range, infinity above it
__device__ __forceinline__ double pow2_biased(int ex) {
    return ex < 1 ? 0.0
                  : (ex > 2046 ? __longlong_as_double(0x7FF0000000000000ll)
                               : __longlong_as_double((long long)ex << 52));
}

// ---- slicing ----------------------------------------------------------------------------
// Biased float64 exponent (0 for zero and subnormal values, which are treated as zero).
__device__ __forceinline__ int bexp(double x) {
    return (int)((__double_as_longlong(x) >> 52) & 0x7FF);
}
// 63-bit fixed-point magnitude of x against the binade 2^{e - 1022} (e >= bexp(x)):
// floor(|x| 2^{63 - (e - 1022)}) = (m << 10) >> (e - bexp(x)), m the 53-bit significand
// with its leading bit; below 2^63.  Branch-free in 32-bit words (zero and subnormal values
// shift out completely).
__device__ __forceinline__ uint64_t fixed63(double x, int e) {
    const uint64_t u = (uint64_t)__double_as_longlong(x);
    const uint32_t hw = (uint32_t)(u >> 32), lw = (uint32_t)u;
    const int ex = (int)((hw >> 20) & 0x7FF);
    uint32_t h = __funnelshift_l(lw, (hw & 0xFFFFFu) | 0x100000u, 10);
    uint32_t l = lw << 10;
    int d = ex == 0 ? 64 : e - ex;
    const bool big = d >= 32;   // a whole word first
    l = big ? h : l;
    h = big ? 0u : h;
    d = big ? d - 32 : d;
    l = __funnelshift_rc(l, h, (uint32_t)d);
    h = d >= 32 ? 0u : (h >> (d & 31));
    return ((uint64_t)h << 32) | l;
}
// bf16 bit pattern of the signed 7-bit slice: the float 2^23 + s (sign folded into the bit
// pattern) plus -+2^23 is exactly +-s; its upper 16 bits are the bf16 value.
__device__ __forceinline__ uint32_t slice_f32_bits(uint32_t s7, uint32_t magic_sign,
                                                   float undo) {
    return __float_as_uint(__uint_as_float((s7 & 127u) | magic_sign) + undo);
}
// slice a (0-based: bits 56 - 7a .. 62 - 7a of F) as a float bit pattern
__device__ __forceinline__ uint32_t slice_bits(uint64_t F, int a, uint32_t ms, float undo) {
    const uint32_t hi = (uint32_t)(F >> 32), lo = (uint32_t)F;
    uint32_t s;
    switch (a) {
        case 0: s = hi >> 24; break;
        case 1: s = hi >> 17; break;
        case 2: s = hi >> 10; break;
        case 3: s = hi >> 3; break;
        case 4: s = __funnelshift_r(lo, hi, 28); break;
        case 5: s = lo >> 21; break;
        case 6: s = lo >> 14; break;
        case 7: s = lo >> 7; break;
        default: s = lo; break;
    }
    return slice_f32_bits(s, ms, undo);
}
__device__ __forceinline__ uint32_t sign_magic(bool neg) {
    return 0x4B000000u | (neg ? 0x80000000u : 0u);
}
__device__ __forceinline__ float sign_undo(bool neg) { return neg ? 8388608.f : -8388608.f; }
// the same -+2^23 from the magic pattern: its sign flipped
__device__ __forceinline__ float undo_of(uint32_t magic_sign) {
    return __uint_as_float(magic_sign ^ 0x80000000u);
}
// two bf16 in one word, first in the low half: the floats hold at most 8 significant bits,
// so the conversion is exact
__device__ __forceinline__ uint32_t pack_bf16(uint32_t f0, uint32_t f1) {
    uint32_t r;
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(__uint_as_float(f1)), "f"(__uint_as_float(f0)));
    return r;
}

// Byte slices (the Gram): slice a (0-based) is byte 7 - a of F (bits 56 - 8a .. 63 - 8a;
// slice 0 below 2^7, the others below 2^8), placed in the low byte of the pattern of the
// float 2^23 (sign folded in) by one byte permutation; adding -+2^23 leaves exactly +-s.
__device__ __forceinline__ uint32_t byte_slice_bits(uint64_t F, int a, uint32_t ms, float undo) {
    const uint32_t hi = (uint32_t)(F >> 32), lo = (uint32_t)F;
    uint32_t w;
    switch (a) {
        case 0: w = __byte_perm(hi, ms, 0x7653); break;
        case 1: w = __byte_perm(hi, ms, 0x7652); break;
        case 2: w = __byte_perm(hi, ms, 0x7651); break;
        case 3: w = __byte_perm(hi, ms, 0x7650); break;
        case 4: w = __byte_perm(lo, ms, 0x7653); break;
        case 5: w = __byte_perm(lo, ms, 0x7652); break;
        case 6: w = __byte_perm(lo, ms, 0x7651); break;
        default: w = __byte_perm(lo, ms, 0x7650); break;
    }
    return __float_as_uint(__uint_as_float(w) + undo);
}
// the eight exact byte-pair group sums G_2 .. G_9 combined into V / 2^14,
// V = sum_g G_g 2^{8(9-g)} (|G_g| < 2^24, |G_2| < 2^21): G_2 2^42 + G_3 2^34 + G_4 2^26 +
// G_5 2^18 + G_6 2^10 + G_7 2^2 + G_8 / 2^6 + G_9 / 2^14, the last two rounded to the
// nearest integer (unbiased), within one unit of V / 2^14, below 2^63.
__device__ __forceinline__ long long combine_byte_groups(const float (&g)[8]) {
    long long acc = (long long)(__float2int_rn(g[1]) * 4 + __float2int_rn(g[0]) * 1024) << 32;
    acc += (long long)__float2int_rn(g[2]) * 67108864;
    acc += (long long)__float2int_rn(g[3]) * 262144;
    acc += (long long)__float2int_rn(g[4]) * 1024;
    return acc + (__float2int_rn(g[5]) * 4 + ((__float2int_rn(g[6]) + 32) >> 6) +
                  ((__float2int_rn(g[7]) + 8192) >> 14));
}

// 16-byte global -> shared copy by this thread (cp.async); src_bytes 0 writes zeros
__device__ __forceinline__ void cp_async16_zfill(void* dst, const void* src, uint32_t src_bytes) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(bulk::smem_addr(dst)),
                 "l"(src), "r"(src_bytes)
                 : "memory");
}

// ---- the update -------------------------------------------------------------------------
// One persistent CTA per SM, warp-specialised:
//   warps 0-7  (slicers): per 128-row tile, take the tile's X values (each thread half a row,
//              P/2 values, copied one tile ahead with cp.async into the thread's own
//              shared chunks), take the row binade, and cut the values into the nine slices,
//              one K-step (16 columns) at a time, into a ring of kStages shared stages;
//   warp 8     (MMA): per K-step one thread issues one MMA per X slice a, against the C
//              slices 1 .. 10 - a stacked along N (N = (10 - a) Q, in pieces of <= 256),
//              starting at the columns of group a + 1, so every pair (a, b) accumulates into
//              group a + b; one of kSets tensor-memory accumulator sets (two when 2 x 9 Q
//              columns fit in 512); each stage is committed back to the slicers and each
//              finished tile to the epilogue;
//   warp 9     (prefetch): while the slicers start tile k it asks L2 for the X and Y rows
//              of tile k + 2 (bulk prefetches), so the slicers' copies and the epilogue's
//              loads find their rows in L2 and HBM streams without gaps;
//   warps 10-17 (epilogue): warp w reads lane quarter w % 4 (32 rows) of the finished set
//              for half of the Q columns ((w - 10) / 4), combines the nine groups, releases
//              the accumulator set, then applies scale and subtraction and writes OUT.
// mbarriers: full[s] / empty[s] per ring stage, acc_full[b] / acc_empty[b] and
// erow_full[b] per accumulator set.  Each wait is bounded; a wait that runs out sets a
// shared abort word that every role checks, so all roles leave their loops.
constexpr int kSlicerWarps = 8;
constexpr int kMmaWarp = 8;
constexpr int kPrefetchWarp = 9;
constexpr int kEpiWarp0 = 10;
constexpr int kEpiWarps = 8;
constexpr int kUpdThreads = (kEpiWarp0 + kEpiWarps) * 32;
constexpr int kPrefetchAhead = 2;   // tiles of lead of the L2 prefetch
constexpr int kKS = 16;          // columns of X per ring stage (one MMA K-step)
constexpr int kStages = 3;

template <int P, int Q>
struct UpdShape {
    static_assert(P % 16 == 0 && P >= 16 && P <= 64, "P: multiple of 16, at most 64");
    static_assert(Q == 16 || Q == 32, "Q: 16 or 32");
    static constexpr int kSliceStage = kTile * kKS * 2;            // one slice of one stage
    static constexpr int kStageBytes = kSlices * kSliceStage;      // 32 KB
    static constexpr int kSliceB = Q * P * 2;                      // one slice of C
    // the nine C slices are stacked along N (B row (b - 1) Q + q), so one MMA of N =
    // (10 - a) Q per X slice a deposits every pair (a, b) into group a + b
    static constexpr int kOffB = kStages * kStageBytes;
    // the next tile's X values, copied by the slicers themselves (cp.async), in chunks of
    // 16 bytes laid out [chunk][slicer thread] so that every access is conflict-free
    static constexpr int kOffRaw = kOffB + kSlices * kSliceB;
    static constexpr int kRawChunks = P / 4;                       // per slicer thread
    static constexpr int kSmem = kOffRaw + kRawChunks * kSlicerWarps * 32 * 16 + 1024;
    static_assert(kSmem <= 232448, "shared memory");
    static constexpr int kLboA = (kTile / 8) * 128;                // next 8 columns of A
    static constexpr int kLboB = (kSlices * Q / 8) * 128;          // next 8 columns of B
    static constexpr uint32_t kAcc = (uint32_t)(kGroups * Q);      // columns of one set
    static constexpr int kSets = 2 * kAcc <= 512 ? 2 : 1;          // accumulator sets
    static constexpr uint32_t kCols = 512;                         // allocated columns
    static constexpr int kKSteps = P / kKS;
};

__device__ __forceinline__ bool wait_or_abort(uint64_t* bar, uint32_t parity,
                                              volatile int* abort) {
    const long long t0 = clock64();
    while (!bulk::mbar_test(bar, parity)) {
        if (*abort) return false;
        if (clock64() - t0 > bulk::kWaitCycles) {
            *abort = 1;
            return false;
        }
    }
    return true;
}
// named barrier `id` over `count` threads that also returns the OR of v over them
__device__ __forceinline__ bool bar_or(int id, int count, bool v) {
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t"
        "setp.ne.u32 p, %1, 0;\n\t"
        "barrier.red.or.pred q, %2, %3, p;\n\t"
        "selp.u32 %0, 1, 0, q;\n\t}"
        : "=r"(r)
        : "r"((uint32_t)v), "r"(id), "r"(count)
        : "memory");
    return r != 0;
}
// hint: bring [p, p + bytes) into L2 (p 16-byte aligned, bytes a multiple of 16)
__device__ __forceinline__ void prefetch_l2(const void* p, uint32_t bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}
// the rows [r0, r0 + rows) of every block of a multi-block operand, into L2
__device__ __forceinline__ void prefetch_rows(const MB<const double>& M, int64_t r0, int64_t rows,
                                              int64_t n) {
    if (r0 >= n) return;
    const int64_t cnt = (r0 + rows <= n ? rows : n - r0) * M.w;
    for (int b = 0; b < M.count; ++b)
        for (int64_t off = 0; off < cnt; off += 8192)   // pieces of at most 64 KB
            prefetch_l2(M.blk(b) + r0 * M.w + off,
                        (uint32_t)((cnt - off < 8192 ? cnt - off : 8192) * sizeof(double)));
}
// The prefetch role: `started` counts the tiles the slicers have begun; whenever it moves,
// ask L2 for the rows of the tile kPrefetchAhead ahead of the newest one.  The prefetch is
// only a hint, so a role that waits too long simply stops.
template <typename F>
__device__ __forceinline__ void prefetch_role(volatile int* started, volatile int* abort,
                                              int my_tiles, int ahead, F issue) {
    for (int d = 0; d < ahead && d < my_tiles; ++d) issue(d);
    int done = 0;
    long long t0 = clock64();
    while (done < my_tiles && !*abort) {
        const int st = *started;
        if (st > done) {
            done = st;
            if (st - 1 + ahead < my_tiles) issue(st - 1 + ahead);
            t0 = clock64();
        } else if (clock64() - t0 > bulk::kWaitCycles) {
            break;
        }
    }
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bulk::smem_addr(bar))
                 : "memory");
}

// OUT = Y - X C (beta_on = 1: the CGS update) or OUT = X C (beta_on = 0: the product with
// R^{-1}) with X = the P columns of X.count blocks (each X.w a multiple of 8), C P x Q
// (row-major, ldc = Q), Y and OUT single n x Q blocks.  OUT may be Y, and OUT may be X
// itself (P = Q, one block): a tile's rows are read by the slicers before the MMAs of that
// tile complete, and written by the epilogue only after.
template <int P, int Q>
__global__ void __launch_bounds__(kUpdThreads, 1)
k_oz_update(MB<const double> X, const double* __restrict__ C, MB<const double> Y,
            MB<double> OUT, int64_t n, int beta_on, int* err) {
    using S = UpdShape<P, Q>;
    extern __shared__ __align__(1024) unsigned char oz_raw[];
    unsigned char* sm = oz_raw + ((1024 - (bulk::smem_addr(oz_raw) & 1023)) & 1023);
    __shared__ __align__(8) uint64_t full[kStages], empty[kStages];
    __shared__ __align__(8) uint64_t acc_full[2], acc_empty[2], erow_full[2], erow_empty[2], fin;
    __shared__ uint32_t tslot;
    __shared__ int erow[2][kTile];
    __shared__ int fcol[Q];
    __shared__ volatile int abort_flag;
    __shared__ volatile int started;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t sA = bulk::smem_addr(sm), sB = sA + S::kOffB;

    if (warp == 0) tmem_alloc(&tslot, S::kCols);
    if (tid == 0) {
        for (int i = 0; i < kStages; ++i) {
            bulk::mbar_init(&full[i], kSlicerWarps);
            bulk::mbar_init(&empty[i], 1);
        }
        for (int b = 0; b < 2; ++b) {
            bulk::mbar_init(&acc_full[b], 1);
            bulk::mbar_init(&acc_empty[b], kEpiWarps);
            bulk::mbar_init(&erow_full[b], kSlicerWarps);
            bulk::mbar_init(&erow_empty[b], kEpiWarps);
        }
        bulk::mbar_init(&fin, 1);
        abort_flag = 0;
        started = 0;
        bulk::fence_barrier_init();
    }
    // C: column binades, then the slices of every entry into the B operand (N = Q x K = P)
    if (tid < Q) {
        int f = 0;
        for (int k = 0; k < P; ++k) f = max(f, bexp(C[(int64_t)k * Q + tid]));
        fcol[tid] = f;
    }
    __syncthreads();
    for (int e = tid; e < P * Q; e += blockDim.x) {
        const int k = e / Q, q = e - k * Q;
        const double c = C[(int64_t)k * Q + q];
        const uint64_t F = fixed63(c, fcol[q]);
        const bool neg = (__double_as_longlong(c) >> 63) != 0;
        const uint32_t ms = sign_magic(neg);
        const float undo = sign_undo(neg);
#pragma unroll
        for (int a = 0; a < kSlices; ++a) {
            const int nrow = a * Q + q;
            const int off = ((k >> 3) * (kSlices * Q / 8) + (nrow >> 3)) * 128 + (nrow & 7) * 16 +
                            (k & 7) * 2;
            *reinterpret_cast<uint16_t*>(sm + S::kOffB + off) =
                (uint16_t)(slice_bits(F, a, ms, undo) >> 16);
        }
    }
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tbase = tslot;
    const int64_t ntiles = (n + kTile - 1) / kTile;

    if (warp < kSlicerWarps) {
        // ---- slicers: thread = (row r, half h); the half holds column groups h + 2j
        const int r = warp * 16 + (lane & 15), h = lane >> 4;
        // this thread's row of a tile, copied one tile ahead into its own 16-byte chunks
        unsigned char* xbuf = sm + S::kOffRaw + tid * 16;
        auto copy_ahead = [&](int64_t tl) {
            if (tl < ntiles) {
                const int64_t i = tl * kTile + r;
#pragma unroll
                for (int j = 0; j < P / 16; ++j) {
                    const int col = (h + 2 * j) * 8, b = col / X.w;
                    const double* src = X.blk(b) + (i < n ? i : 0) * X.w + (col - b * X.w);
#pragma unroll
                    for (int u = 0; u < 4; ++u)
                        cp_async16_zfill(xbuf + (j * 4 + u) * (kSlicerWarps * 32 * 16),
                                         src + 2 * u, i < n ? 16u : 0u);
                }
            }
            asm volatile("cp.async.commit_group;" ::: "memory");
        };
        copy_ahead(blockIdx.x);
        int stage = 0;
        int lt = 0;
        for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++lt) {
            const int buf = lt & 1;   // row-binade buffer (two tiles in flight)
            if (lt >= 2 && !wait_or_abort(&erow_empty[buf], ((lt >> 1) - 1) & 1, &abort_flag))
                break;
            if (tid == 0) started = lt + 1;
            double xv[P / 2];
            asm volatile("cp.async.wait_group 0;" ::: "memory");
#pragma unroll
            for (int j = 0; j < P / 16; ++j)
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const double2 v = *reinterpret_cast<const double2*>(
                        xbuf + (j * 4 + u) * (kSlicerWarps * 32 * 16));
                    xv[j * 8 + 2 * u] = v.x;
                    xv[j * 8 + 2 * u + 1] = v.y;
                }
            copy_ahead(tile + gridDim.x);   // lands while this tile is cut
            int e = 0;
#pragma unroll
            for (int u = 0; u < P / 2; ++u) e = max(e, bexp(xv[u]));
            e = max(e, __shfl_xor_sync(0xffffffffu, e, 16));
            if (h == 0) erow[buf][r] = e;
            __syncwarp();
            if (lane == 0) mbar_arrive(&erow_full[buf]);
            bool ok = true;
#pragma unroll
            for (int j = 0; j < P / 16; ++j) {
                // K-step j = column groups 2j, 2j+1; this thread holds group 2j + h
                const int slot = stage % kStages, use = stage / kStages;
                if (use >= 1 && !wait_or_abort(&empty[slot], (use - 1) & 1, &abort_flag)) {
                    ok = false;
                    break;
                }
                uint64_t F[8];
                uint32_t ms[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const double x = xv[j * 8 + u];
                    F[u] = fixed63(x, e);
                    const bool neg = (__double_as_longlong(x) >> 63) != 0;
                    ms[u] = sign_magic(neg);
                }
                unsigned char* dst = sm + slot * S::kStageBytes +
                                     (h * (kTile / 8) + (r >> 3)) * 128 + (r & 7) * 16;
#pragma unroll
                for (int a = 0; a < kSlices; ++a) {
                    uint4 v;
                    v.x = pack_bf16(slice_bits(F[0], a, ms[0], undo_of(ms[0])),
                                    slice_bits(F[1], a, ms[1], undo_of(ms[1])));
                    v.y = pack_bf16(slice_bits(F[2], a, ms[2], undo_of(ms[2])),
                                    slice_bits(F[3], a, ms[3], undo_of(ms[3])));
                    v.z = pack_bf16(slice_bits(F[4], a, ms[4], undo_of(ms[4])),
                                    slice_bits(F[5], a, ms[5], undo_of(ms[5])));
                    v.w = pack_bf16(slice_bits(F[6], a, ms[6], undo_of(ms[6])),
                                    slice_bits(F[7], a, ms[7], undo_of(ms[7])));
                    *reinterpret_cast<uint4*>(dst + a * S::kSliceStage) = v;
                }
                fence_async_smem();
                __syncwarp();
                if (lane == 0) mbar_arrive(&full[slot]);
                ++stage;
            }
            if (!ok) break;
        }
        asm volatile("cp.async.wait_group 0;" ::: "memory");   // no copy outlives the CTA
    } else if (warp == kMmaWarp) {
        // ---- MMA issue (one thread)
        if (lane == 0) {
            int stage = 0;
            int lt = 0;
            for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++lt) {
                const int set = lt % S::kSets, use = lt / S::kSets;
                if (use >= 1 && !wait_or_abort(&acc_empty[set], (use - 1) & 1, &abort_flag))
                    break;
                tc_fence_after();
                const uint32_t dacc = tbase + (uint32_t)set * S::kAcc;
                bool ok = true;
                for (int j = 0; j < S::kKSteps; ++j) {
                    const int slot = stage % kStages, use = stage / kStages;
                    if (!wait_or_abort(&full[slot], use & 1, &abort_flag)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
#pragma unroll
                    for (int a = 1; a <= kSlices; ++a) {
                        // X slice a times C slices 1 .. 10 - a (B rows 0 .. (10 - a) Q): pair
                        // (a, b) lands in the columns of group a + b; N in pieces of <= 256
                        const uint64_t ad = smem_desc(
                            sA + slot * S::kStageBytes + (a - 1) * S::kSliceStage, S::kLboA, 128);
                        const int na = (kGroups + 1 - a) * Q;
#pragma unroll
                        for (int n0 = 0; n0 < na; n0 += kMaxN) {
                            const int nn = (na - n0) < kMaxN ? (na - n0) : kMaxN;
                            const uint64_t bd = smem_desc(
                                sB + j * 2 * S::kLboB + (n0 / 8) * 128, S::kLboB, 128);
                            mma_bf16(dacc + (uint32_t)((a - 1) * Q + n0), ad, bd,
                                     idesc_bf16_f32(kTile, nn), (j > 0 || a > 1) ? 1u : 0u);
                        }
                    }
                    mma_commit(&empty[slot]);
                    ++stage;
                }
                if (!ok) break;
                mma_commit(&acc_full[set]);
            }
            // every MMA issued has completed before the tensor memory is released
            mma_commit(&fin);
            bulk::mbar_wait(&fin, 0);
        }
        __syncwarp();
    } else if (warp == kPrefetchWarp) {
        if (lane == 0) {
            const int my_tiles = (int)((ntiles - blockIdx.x + gridDim.x - 1) / gridDim.x);
            prefetch_role(&started, &abort_flag, my_tiles, kPrefetchAhead, [&](int lt) {
                const int64_t r0 = (blockIdx.x + (int64_t)lt * gridDim.x) * kTile;
                prefetch_rows(X, r0, kTile, n);
                if (beta_on) prefetch_rows(Y, r0, kTile, n);
            });
        }
        __syncwarp();
    } else {
        // ---- epilogue: quarter qd = warp % 4, rows 32 qd + lane of the tile, columns
        //      c0 .. c0 + Q / 2 - 1
        constexpr int QH = Q / 2;
        const int qd = warp & 3;
        const int m = qd * 32 + lane;
        const int c0 = ((warp - kEpiWarp0) >> 2) * QH;
        int lt = 0;
        for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++lt) {
            const int buf = lt & 1, set = lt % S::kSets;
            const int64_t ri = tile * kTile + m;
            if (!wait_or_abort(&acc_full[set], (lt / S::kSets) & 1, &abort_flag)) break;
            if (!wait_or_abort(&erow_full[buf], (lt >> 1) & 1, &abort_flag)) break;
            tc_fence_after();
            const int er = erow[buf][m];
            __syncwarp();
            if (lane == 0) mbar_arrive(&erow_empty[buf]);
            const uint32_t taddr = tbase + ((uint32_t)(qd * 32) << 16) + (uint32_t)set * S::kAcc +
                                   (uint32_t)c0;
            long long V[QH];
#pragma unroll
            for (int k = 0; k < QH; k += 2) {
                float g[kGroups][2];
#pragma unroll
                for (int gi = 0; gi < kGroups; ++gi)
                    tmem_ld2(taddr + (uint32_t)(gi * Q + k), g[gi]);
                tmem_wait_ld();
#pragma unroll
                for (int u = 0; u < 2; ++u) {
                    float gu[kGroups];
#pragma unroll
                    for (int gi = 0; gi < kGroups; ++gi) gu[gi] = g[gi][u];
                    V[k + u] = combine_groups(gu);
                }
            }
            // the accumulator is read: the MMA warp may start the next tile in it
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&acc_empty[set]);
            if (ri < n) {
#pragma unroll
                for (int k = 0; k < QH; k += 4) {
                    double yv[4] = {0.0, 0.0, 0.0, 0.0};
                    if (beta_on) {
                        const double2* yr =
                            reinterpret_cast<const double2*>(Y.blk(0) + ri * Y.w + c0 + k);
                        const double2 a = yr[0], b = yr[1];
                        yv[0] = a.x;
                        yv[1] = a.y;
                        yv[2] = b.x;
                        yv[3] = b.y;
                    }
                    double ov[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const long long v = V[k + u];
                        const double scale = pow2_biased(er + fcol[c0 + k + u] - 1077);
                        ov[u] = fma((double)(beta_on ? -v : v), scale, yv[u]);
                    }
                    double2* orow = reinterpret_cast<double2*>(OUT.blk(0) + ri * OUT.w + c0 + k);
                    orow[0] = make_double2(ov[0], ov[1]);
                    orow[1] = make_double2(ov[2], ov[3]);
                }
            }
        }
    }
    __syncthreads();
    if (abort_flag && tid == 0) atomicOr(err, 4);
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc(tbase, S::kCols);
    }
}

// ---- the Gram product ---------------------------------------------------------------
// C = X^T Y over the n rows (CGS coefficients Q^T (A W), the A-CholQR Gram W^T (A W)):
// X n x P (P <= 64), Y n x Q (Q = 16 or 32).  The contraction runs over rows, in tiles of 64
// rows: every column of X and of Y is scaled by its binade over the tile (e_p, f_q), and
// cut into eight byte slices of the same 63-bit fixed-point magnitude F (slice a, 1-based,
// holds bits 64 - 8a .. 71 - 8a; bf16 holds every byte exactly).  The 36 slice pairs with
// a + b <= 9 form eight groups g = 2..9; the epilogue adds the tile's
// (V / 2^14) 2^{e_p + f_q - 2100}, V = sum_g G_g 2^{8(9-g)}, into a float64 accumulator per
// output held in registers across the CTA's tiles (the dropped pairs and the truncation of
// F weigh at most about 2^-60 of the product of the column maxima per term).  Each CTA
// writes its P x Q partial sum; k_gram_reduce adds the partials in CTA order.
//
// Slice pairs in M: the A operand of one MMA holds two X slices, a (rows 0-63, X column p
// in row p) and a + 1 (rows 64-127), so every MMA runs at M = 128.  The MMA of the pair
// (a, a + 1), a odd, multiplies by the Y slices 1 .. 9 - a stacked along N and starts at
// the accumulator columns of group a + 1: tensor-memory lanes 0-63 receive the pairs (a, b)
// in the columns of group a + b, lanes 64-127 the pairs (a + 1, b) in the columns of group
// a + b as well, that is group (a + 1 + b) - 1.  So column block j holds group j + 2 in the
// upper lanes and group j + 3 in the lower lanes (block 7 of the lower lanes, group 10, is
// beyond the 36 pairs and not read).  A group of one half holds at most four pairs, so its
// fp32 sum stays exact (4 x 64 rows x 255^2 < 2^24).  Four MMAs per K-step; an accumulator
// set is 8 Q columns, so two sets fit in tensor memory and the MMAs of one tile overlap the
// epilogue of the previous one.
//
//   warps 0-7  (slicers): warp w cuts row group w of the tile (rows 8 w .. 8 w + 7), lane =
//              column within each 32-column block of X | Y; pass 1 takes the column
//              binades of the tile (per-warp maxima in shared memory, then the max over the
//              eight row groups), pass 2 writes the warp's 8 rows of every slice into the
//              stage of its K-step (w / 2), K-group w % 2.  Two slicer warps per SM
//              sub-partition;
//   warp 8     (MMA): per K-step the four pair MMAs (M = 128, K = 16, N in pieces <= 256);
//   warp 9     (producer): one thread copies the tile's rows of every X block and of Y
//              (contiguous runs of 64 x w doubles) into one of two raw shared buffers with
//              bulk copies completing on an mbarrier, one tile ahead of the slicers;
//   warps 10-17 (epilogue): warp w reads lane quarter q = w % 4 of the accumulator, for
//              the columns of half (w - 10) / 4 of C; the thread for output row
//              p = 32 (q & 1) + lane holds the upper groups (q < 2, lanes 0-63) or the lower
//              groups (q >= 2, lanes 64-127) of that row.  It combines its groups of its
//              Q / 2 columns, releases the accumulator to the MMA warp, then converts and
//              scales them into float64 accumulators of its own; the upper and lower
//              accumulators of an output are added once, at the end.
constexpr int kGramSlicers = 8;
constexpr int kGramMmaWarp = 8;
constexpr int kGramProducerWarp = 9;
constexpr int kGramEpiWarp0 = 10;
constexpr int kGramEpiWarps = 8;
constexpr int kGramThreads = (kGramEpiWarp0 + kGramEpiWarps) * 32;
constexpr int kGramCexp = 3;         // tile binade buffers (the epilogue frees one late)
constexpr int kGramRows = 64;        // rows per tile (binade scope, exact fp32 sums)
constexpr int kGramStages = 4;      // one tile of K-steps: no stage is reused within a tile
constexpr int kGSlices = 8;          // byte slices of the 63-bit fixed-point magnitude
constexpr int kGGroups = 8;          // byte-pair groups g = a + b = 2..9
constexpr int kPairs = kGSlices / 2; // X slice pairs per K-step

template <int P, int Q>
struct GramShape {
    static_assert(P % 16 == 0 && P >= 16 && P <= 64, "P: multiple of 16, at most 64");
    static_assert(Q == 16 || Q == 32, "Q: 16 or 32");
    static constexpr int kM = 128;                                 // MMA M (slice pair)
    static constexpr int kPairA = kM * kKS * 2;                    // 4 KB: one slice pair
    static constexpr int kSliceB = Q * kKS * 2;
    static constexpr int kStageBytes = kPairs * kPairA + kGSlices * kSliceB;
    static constexpr int kOffB = kPairs * kPairA;                  // B inside a stage
    static constexpr int kRawX = kGramRows * P * 8;                // raw X tile, bytes
    static constexpr int kRawY = kGramRows * Q * 8;
    static constexpr int kOffRaw = kGramStages * kStageBytes;      // raw buffers after ring
    static constexpr int kSmem = kOffRaw + 2 * (kRawX + kRawY) + 1024;
    static constexpr int kLboA = (kM / 8) * 128;                   // 2 KB
    static constexpr int kLboB = (kGSlices * Q / 8) * 128;         // Y slices stacked in N
    static constexpr uint32_t kAcc = (uint32_t)(kGGroups * Q);
    static constexpr int kSets = 2 * kAcc <= 512 ? 2 : 1;          // accumulator sets
    static_assert(kSets == 2, "two accumulator sets");
    static constexpr uint32_t kCols = 512;
    static constexpr int kT = P + Q;                               // columns sliced per row
    static constexpr int kNB = (kT + 31) / 32;                     // column blocks
    static constexpr int kKSteps = kGramRows / kKS;                // 4
    static_assert(kKSteps * 2 == kGramSlicers, "one slicer warp per 8-row group");
    static_assert(kSmem <= 232448, "shared memory");
};

// partials[cta * 4096 + p * Q + q] = this CTA's share of (X^T Y)[p, q]
template <int P, int Q>
__global__ void __launch_bounds__(kGramThreads, 1)
k_oz_gram(MB<const double> X, MB<const double> Y, int64_t n, double* __restrict__ partials,
          int* err) {
    using S = GramShape<P, Q>;
    constexpr int QH = Q / 2;
    extern __shared__ __align__(1024) unsigned char oz_raw[];
    unsigned char* sm = oz_raw + ((1024 - (bulk::smem_addr(oz_raw) & 1023)) & 1023);
    __shared__ __align__(8) uint64_t full[kGramStages], empty[kGramStages];
    __shared__ __align__(8) uint64_t acc_full[2], acc_empty[2], fin;
    __shared__ __align__(8) uint64_t cexp_full[kGramCexp], cexp_empty[kGramCexp];
    __shared__ __align__(8) uint64_t raw_full[2], raw_empty[2];
    __shared__ uint32_t tslot;
    __shared__ int cexp[kGramCexp][S::kT];            // tile binades: X columns, then Y
    __shared__ int cmax[kGramSlicers][S::kNB * 32];   // per row group, pass 1
    __shared__ volatile int abort_flag;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t sbase = bulk::smem_addr(sm);
    double* rawx[2] = {reinterpret_cast<double*>(sm + S::kOffRaw),
                       reinterpret_cast<double*>(sm + S::kOffRaw + S::kRawX)};
    double* rawy[2] = {reinterpret_cast<double*>(sm + S::kOffRaw + 2 * S::kRawX),
                       reinterpret_cast<double*>(sm + S::kOffRaw + 2 * S::kRawX + S::kRawY)};

    if (warp == 0) tmem_alloc(&tslot, S::kCols);
    if (tid == 0) {
        for (int i = 0; i < kGramStages; ++i) {
            bulk::mbar_init(&full[i], 2);            // the two row groups of a K-step
            bulk::mbar_init(&empty[i], 1);
        }
        for (int b = 0; b < 2; ++b) {
            bulk::mbar_init(&acc_full[b], 1);
            bulk::mbar_init(&acc_empty[b], kGramEpiWarps);
            bulk::mbar_init(&raw_full[b], 1);
            bulk::mbar_init(&raw_empty[b], kGramSlicers);
        }
        for (int b = 0; b < kGramCexp; ++b) {
            bulk::mbar_init(&cexp_full[b], kGramSlicers);
            bulk::mbar_init(&cexp_empty[b], kGramEpiWarps);
        }
        bulk::mbar_init(&fin, 1);
        abort_flag = 0;
        bulk::fence_barrier_init();
    }
    // the ring starts zeroed: rows p >= P of each half and the half of slice 10 stay zero
    for (int e = tid * 16; e < kGramStages * S::kStageBytes; e += blockDim.x * 16)
        *reinterpret_cast<uint4*>(sm + e) = make_uint4(0u, 0u, 0u, 0u);
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tbase = tslot;
    const int64_t ntiles = (n + kGramRows - 1) / kGramRows;

    if (warp < kGramSlicers) {
        // ---- slicers: rows 8 rg .. 8 rg + 7 of the tile; column 32 cb + lane of X | Y
        const int rg = warp, ks = rg >> 1, par = rg & 1;
        int raw_off[S::kNB], wcol[S::kNB];
        bool act[S::kNB], isxc[S::kNB];
#pragma unroll
        for (int cb = 0; cb < S::kNB; ++cb) {
            const int c = cb * 32 + lane;
            act[cb] = c < S::kT;
            isxc[cb] = c < P;
            const int cc = isxc[cb] ? c : c - P;
            const int w = isxc[cb] ? X.w : Q;
            const int blk = (act[cb] && isxc[cb]) ? cc / X.w : 0;
            const int cw = act[cb] ? cc - blk * w : 0;
            // raw element (row, column) = raw[blk * 64 * w + row * w + cw]
            raw_off[cb] = blk * kGramRows * w + cw + 8 * rg * w;
            wcol[cb] = w;
        }
        int lt = 0;
        bool failed = false;   // the slicer warps leave together (they share named barriers)
        for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++lt) {
            const int buf = lt & 1;                    // raw buffer (two tiles in flight)
            const int cb3 = lt % kGramCexp;            // binade buffer
            if (lt >= kGramCexp && !failed &&
                !wait_or_abort(&cexp_empty[cb3], ((lt / kGramCexp) - 1) & 1, &abort_flag))
                failed = true;
            if (!failed && !wait_or_abort(&raw_full[buf], (lt >> 1) & 1, &abort_flag))
                failed = true;
            if (bar_or(1, kGramSlicers * 32, failed || abort_flag)) break;
            const int64_t r0 = tile * kGramRows;
            const int rows = (int)((n - r0) < kGramRows ? (n - r0) : kGramRows);
            const int myrows = rows - 8 * rg;            // rows of this group (may be <= 0)
            // pass 1: binade of each column over this row group, then over the tile
            int e[S::kNB];
#pragma unroll
            for (int cb = 0; cb < S::kNB; ++cb) {
                const double* raw = (isxc[cb] ? rawx[buf] : rawy[buf]) + raw_off[cb];
                int m = 0;
                if (act[cb]) {
#pragma unroll
                    for (int u = 0; u < 8; ++u)
                        if (u < myrows) m = max(m, bexp(raw[u * wcol[cb]]));
                }
                cmax[rg][cb * 32 + lane] = m;
            }
            asm volatile("bar.sync 1, %0;" ::"r"(kGramSlicers * 32) : "memory");
#pragma unroll
            for (int cb = 0; cb < S::kNB; ++cb) {
                int m = 0;
#pragma unroll
                for (int r = 0; r < kGramSlicers; ++r) m = max(m, cmax[r][cb * 32 + lane]);
                e[cb] = m;
                if (rg == 0 && act[cb]) cexp[cb3][cb * 32 + lane] = m;
            }
            asm volatile("bar.sync 1, %0;" ::"r"(kGramSlicers * 32) : "memory");
            __syncwarp();
            if (lane == 0) mbar_arrive(&cexp_full[cb3]);
            // pass 2: this row group's 8 rows of every slice, into the stage of K-step ks
            const int stage = lt * S::kKSteps + ks;
            const int slot = stage % kGramStages, use = stage / kGramStages;
            if (use >= 1 && !wait_or_abort(&empty[slot], (use - 1) & 1, &abort_flag))
                failed = true;
            if (!failed) {
                unsigned char* st = sm + slot * S::kStageBytes;
#pragma unroll
                for (int cb = 0; cb < S::kNB; ++cb) {
                    if (!act[cb]) continue;
                    const double* raw = (isxc[cb] ? rawx[buf] : rawy[buf]) + raw_off[cb];
                    const int cc = isxc[cb] ? cb * 32 + lane : cb * 32 + lane - P;
                    uint64_t F[8];
                    uint32_t ms[8];
#pragma unroll
                    for (int u = 0; u < 8; ++u) {
                        const double x = (u < myrows) ? raw[u * wcol[cb]] : 0.0;
                        F[u] = fixed63(x, e[cb]);
                        const bool neg = (__double_as_longlong(x) >> 63) != 0;
                        ms[u] = sign_magic(neg);
                    }
#pragma unroll
                    for (int a = 0; a < kGSlices; ++a) {
                        uint4 v;
                        v.x = pack_bf16(byte_slice_bits(F[0], a, ms[0], undo_of(ms[0])),
                                        byte_slice_bits(F[1], a, ms[1], undo_of(ms[1])));
                        v.y = pack_bf16(byte_slice_bits(F[2], a, ms[2], undo_of(ms[2])),
                                        byte_slice_bits(F[3], a, ms[3], undo_of(ms[3])));
                        v.z = pack_bf16(byte_slice_bits(F[4], a, ms[4], undo_of(ms[4])),
                                        byte_slice_bits(F[5], a, ms[5], undo_of(ms[5])));
                        v.w = pack_bf16(byte_slice_bits(F[6], a, ms[6], undo_of(ms[6])),
                                        byte_slice_bits(F[7], a, ms[7], undo_of(ms[7])));
                        // X: slice a (0-based) in pair a / 2, rows 64 (a % 2) + cc, K-group
                        // par; Y: slice a is B rows a Q .. a Q + Q - 1
                        const int off =
                            isxc[cb] ? (a >> 1) * S::kPairA + par * S::kLboA +
                                           ((64 * (a & 1) + cc) >> 3) * 128 + (cc & 7) * 16
                                     : S::kOffB + par * S::kLboB + ((a * Q + cc) >> 3) * 128 +
                                           (cc & 7) * 16;
                        *reinterpret_cast<uint4*>(st + off) = v;
                    }
                }
                fence_async_smem();
                __syncwarp();
                if (lane == 0) mbar_arrive(&full[slot]);
            }
            // the raw buffer may be refilled
            __syncwarp();
            if (lane == 0) mbar_arrive(&raw_empty[buf]);
        }
    } else if (warp == kGramProducerWarp) {
        if (lane == 0) {
            int lt = 0;
            for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++lt) {
                const int buf = lt & 1;
                if (lt >= 2 && !wait_or_abort(&raw_empty[buf], ((lt >> 1) - 1) & 1, &abort_flag))
                    break;
                const int64_t r0 = tile * kGramRows;
                const int rows = (int)((n - r0) < kGramRows ? (n - r0) : kGramRows);
                const uint32_t bx = (uint32_t)rows * X.w * 8, by = (uint32_t)rows * Q * 8;
                bulk::mbar_expect_tx(&raw_full[buf], bx * X.count + by);
                for (int b = 0; b < X.count; ++b)
                    bulk::bulk_g2s(rawx[buf] + b * kGramRows * X.w, X.blk(b) + r0 * X.w, bx,
                                   &raw_full[buf]);
                bulk::bulk_g2s(rawy[buf], Y.blk(0) + r0 * Q, by, &raw_full[buf]);
            }
            // every copy issued has landed before the CTA exits
            if (lt > 0) bulk::mbar_wait(&raw_full[(lt - 1) & 1], ((lt - 1) >> 1) & 1);
        }
        __syncwarp();
    } else if (warp == kGramMmaWarp) {
        if (lane == 0) {
            int stage = 0;
            int lt = 0;
            for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++lt) {
                const int set = lt % S::kSets, use = lt / S::kSets;
                if (use >= 1 && !wait_or_abort(&acc_empty[set], (use - 1) & 1, &abort_flag))
                    break;
                tc_fence_after();
                const uint32_t dacc = tbase + (uint32_t)set * S::kAcc;
                bool ok = true;
                for (int ks = 0; ks < S::kKSteps; ++ks) {
                    const int slot = stage % kGramStages, use = stage / kGramStages;
                    if (!wait_or_abort(&full[slot], use & 1, &abort_flag)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t st = sbase + slot * S::kStageBytes;
#pragma unroll
                    for (int j = 0; j < kPairs; ++j) {
                        const int a = 2 * j + 1;                  // 1-based upper slice
                        const uint64_t ad = smem_desc(st + j * S::kPairA, S::kLboA, 128);
                        const int na = (kGSlices + 1 - a) * Q;   // Y slices 1 .. 9 - a
#pragma unroll
                        for (int n0 = 0; n0 < na; n0 += kMaxN) {
                            const int nn = (na - n0) < kMaxN ? (na - n0) : kMaxN;
                            const uint64_t bd =
                                smem_desc(st + S::kOffB + (n0 / 8) * 128, S::kLboB, 128);
                            mma_bf16(dacc + (uint32_t)((a - 1) * Q + n0), ad, bd,
                                     idesc_bf16_f32(S::kM, nn), (ks > 0 || j > 0) ? 1u : 0u);
                        }
                    }
                    mma_commit(&empty[slot]);
                    ++stage;
                }
                if (!ok) break;
                mma_commit(&acc_full[set]);
            }
            mma_commit(&fin);
            bulk::mbar_wait(&fin, 0);
        }
        __syncwarp();
    } else if (warp >= kGramEpiWarp0) {
        // ---- epilogue: row p = 32 (qd & 1) + lane; upper groups (qd < 2) or lower (qd >= 2);
        //      columns c0 .. c0 + QH - 1
        const int qd = warp & 3;
        const bool upper = qd < 2;
        const int p = (qd & 1) * 32 + lane;
        const bool own = p < P;
        const int c0 = ((warp - kGramEpiWarp0) >> 2) * QH;
        const uint32_t lane_base = tbase + ((uint32_t)(qd * 32) << 16) + (uint32_t)c0;
        double acc[QH];
#pragma unroll
        for (int q = 0; q < QH; ++q) acc[q] = 0.0;
        int lt = 0;
        for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++lt) {
            const int set = lt % S::kSets, cb3 = lt % kGramCexp;
            if (!wait_or_abort(&acc_full[set], (lt / S::kSets) & 1, &abort_flag)) break;
            if (!wait_or_abort(&cexp_full[cb3], (lt / kGramCexp) & 1, &abort_flag)) break;
            tc_fence_after();
            const uint32_t taddr = lane_base + (uint32_t)set * S::kAcc;
            // block j holds group j + 2 in the upper lanes and group j + 3 in the lower ones
            long long V[QH];
#pragma unroll
            for (int k = 0; k < QH; k += 2) {
                float g[kGGroups][2];
                if (upper) {
#pragma unroll
                    for (int j = 0; j < kGGroups; ++j)
                        tmem_ld2(taddr + (uint32_t)(j * Q + k), g[j]);
                } else {
#pragma unroll
                    for (int u = 0; u < 2; ++u) g[0][u] = 0.f;
#pragma unroll
                    for (int j = 0; j + 1 < kGGroups; ++j)
                        tmem_ld2(taddr + (uint32_t)(j * Q + k), g[j + 1]);
                }
                tmem_wait_ld();
#pragma unroll
                for (int u = 0; u < 2; ++u) {
                    float gu[kGGroups];
#pragma unroll
                    for (int gi = 0; gi < kGGroups; ++gi) gu[gi] = g[gi][u];
                    V[k + u] = combine_byte_groups(gu);
                }
            }
            // the accumulator is read: the MMA warp may start the next tile in it
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&acc_empty[set]);
            const int ep = own ? cexp[cb3][p] : 0;
#pragma unroll
            for (int q = 0; q < QH; ++q)
                acc[q] = fma((double)V[q], pow2_biased(ep + cexp[cb3][P + c0 + q] - 1077), acc[q]);
            __syncwarp();
            if (lane == 0) mbar_arrive(&cexp_empty[cb3]);
        }
        // upper + lower accumulators of each output, through the (now idle) raw buffers:
        // every tile's copies have landed and been cut before its accumulator was final
        double* red = reinterpret_cast<double*>(sm + S::kOffRaw);   // [64 rows][Q]
        if (!upper) {
#pragma unroll
            for (int q = 0; q < QH; ++q) red[p * Q + c0 + q] = acc[q];
        }
        asm volatile("bar.sync 2, %0;" ::"r"(kGramEpiWarps * 32) : "memory");
        if (upper && own) {
            double* out = partials + (int64_t)blockIdx.x * 4096 + p * Q + c0;
#pragma unroll
            for (int q = 0; q < QH; ++q) out[q] = acc[q] + red[p * Q + c0 + q];
        }
    }
    __syncthreads();
    if (abort_flag && tid == 0) atomicOr(err, 4);
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc(tbase, S::kCols);
    }
}

}  // namespace oz
}  // namespace ekcg
