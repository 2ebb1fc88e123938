// Split-precision (Ozaki-style BF16 slices) GEMM: constants, descriptors and launchers.
#pragma once
#include <cstdint>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "lx_internal.cuh"

namespace lx {

constexpr int SPLIT_NSLICE = 6;                      // digits per FP64 value
constexpr int SPLIT_BETA = 8;                        // bits per digit
constexpr int SPLIT_W = SPLIT_NSLICE * SPLIT_BETA;   // fixed-point bits kept (48)
constexpr int SPLIT_KB = 32;                         // K block (elements) of one pipeline stage
constexpr int SPLIT_TA = 128;                        // A row tile = MMA M
constexpr int SPLIT_TB = 32;                         // largest B row tile (2 sets x 6 diagonals x 32 TMEM columns)
constexpr int SPLIT_SEG_KB = 4;                      // K blocks accumulated in TMEM between int64 drains

// Exponent of an all-zero row segment (below any real exponent; its digits are zero).
constexpr int SPLIT_EXP_NONE = -(1 << 29);

// One matrix whose rows are split: src at (double*)base + src_off, row stride ld.  Before
// splitting, column k is multiplied by 2^(shift_sign * shift[k]) (exact; shift_off < 0: none).
// fixed = 0: each row gets its own power of two (|x| < 2^e over the row: an exponent pass, then
// a digit pass); fixed = 1: the scaled values are known to lie in (-1, 1) and every row takes
// e = 0 (one pass, no maximum); fixed = 2: each row and segment of SPLIT_SEG_KB K blocks (128
// columns) gets its own power of two, int[row][nseg] (SPLIT_EXP_NONE for a zero segment), so
// every value is read once.
struct SplitRowsDesc {
    int64_t src_off;    // doubles
    int64_t dig_off;    // bytes from the workspace base
    int64_t exp_off;    // bytes from the workspace base (int per padded row, times nseg if fixed = 2)
    int64_t shift_off;  // bytes from the workspace base (int per column), or -1
    int ld, rows, K, T, nkb, shift_sign, fixed, nseg;
    int nd, pad;  // digit slices written (the first nd of the block's NSLICE)
};
__host__ __device__ inline int split_nseg(int nkb) { return (nkb + SPLIT_SEG_KB - 1) / SPLIT_SEG_KB; }

// Per-quartet split operands of the two GEMMs.  Column k of H_bra is scaled by 2^-c1[k] into
// (-1, 1) and column k of [p|q]^T by 2^c1[k] (the product is unchanged); likewise H_ket and
// [ab|q] with c2.  Every operand carries one exponent per row.
struct SplitQuartet {
    int64_t a1_dig, a1_exp;  // [p|q]^T rows (Kket Nq), K = Kbra Np, columns scaled by 2^c1
    int64_t b1_dig, b1_exp;  // H_bra rows (nab), columns scaled by 2^-c1
    int64_t a2_dig, a2_exp;  // [ab|q] rows (nab), K = Kket Nq, columns scaled by 2^c2
    int64_t b2_dig, b2_exp;  // H_ket rows (ncd), columns scaled by 2^-c2
    int64_t c1_off, c2_off;  // int[Kbra Np], int[Kket Nq]
    int64_t gidx_off;        // this class's block of the [p+q] index table (gidx_offset)
    int nkb1, nkb2;
    int nd, pad;  // digit slices written (the first nd of the block's NSLICE)
};

// Index table of the [p|q] gathers: for l_bra, l_ket <= 2 LMAX, entry gidx_offset(l_bra,
// l_ket) + q gidx_ld(l_bra) + p holds hidx(p + q) (the position of [p+q]^(0) in the [r]^(0)
// vector of the quartet) as a 16-bit integer, for q < pyr(l_ket), p < pyr(l_bra); rows are
// padded to a multiple of 8 entries so that 8 consecutive entries are one 16-byte load.
constexpr int GIDX_L = 2 * LMAX + 1;  // l_bra (and l_ket) = 0 .. 2 LMAX
__host__ __device__ inline int gidx_ld(int lbra) { return (pyr(lbra) + 7) / 8 * 8; }
__host__ __device__ inline int64_t gidx_offset(int lbra, int lket) {
    int64_t off = 0;
    for (int b = 0; b < GIDX_L; ++b)
        for (int k = 0; k < GIDX_L; ++k) {
            if (b == lbra && k == lket) return off;
            off += (int64_t)pyr(k) * gidx_ld(b);
        }
    return off;  // total size
}
static_assert(NHERM_TOT < 65536, "[r]^(0) positions fit 16 bits");

// D = A B^T: A digits (row tiles of SPLIT_TA), B digits (row tiles of tb = split_tb(N)), both
// with nkb K blocks; D written to (double*)C + c_off with row stride ldc (transpose: D[m][n] ->
// C[n][m]).  B carries one exponent per row; A one per row (a_nseg = 1) or one per row and
// segment of SPLIT_SEG_KB K blocks (a_nseg = split_nseg(nkb), int[row][a_nseg]).  The A operand
// is read only up to M rows rounded to 8 (the last row tile is loaded that far).  B rows past
// N (in its last row tile) may hold anything: they reach only output columns >= N, which are
// dropped.  Only the first nd (4..6) digit slices of each operand are used: the products with
// s + t < nd.
struct SplitGemmDesc {
    int64_t a_dig, a_exp, b_dig, b_exp;
    int64_t c_off;
    int M, N, nkb, ldc, transpose, tb;
    int a_nseg, nd;
};
constexpr int SPLIT_MIN_DIGITS = 4;

// B row tile for an operand of N rows: as few tiles as SPLIT_TB rows allow, each a multiple
// of 16 rows (169 rows -> 6 tiles of 32, 81 -> 3 of 32, 13 -> 1 of 16).
__host__ __device__ inline int split_tb(int N) {
    const int tiles = (N + SPLIT_TB - 1) / SPLIT_TB;
    const int t = (N + tiles - 1) / tiles;
    return (t + 15) / 16 * 16;
}

__host__ __device__ inline int split_rowpad(int rows, int T) { return (rows + T - 1) / T * T; }
__host__ __device__ inline int split_nkb(int K) { return (K + SPLIT_KB - 1) / SPLIT_KB; }
// bytes of the digit planes of an operand (rows padded to T, K padded to SPLIT_KB)
__host__ __device__ inline int64_t split_dig_bytes(int rows, int K, int T) {
    return (int64_t)split_rowpad(rows, T) * split_nkb(K) * SPLIT_KB * SPLIT_NSLICE * 2;
}

cudaError_t init_split_kernels(const int* host_tuv);
cudaError_t launch_split_rows(const SplitRowsDesc* descs, const WorkItem* items, int nitems, const double* src_base,
                              char* ws, cudaStream_t st);
// split_r items and split_rows items in one launch (8 items per block, kinds alternating)
cudaError_t launch_split_operands(const DQuartet* qd, const SplitQuartet* sq, const WorkItem* items_r, int n_r,
                                  const SplitRowsDesc* descs, const WorkItem* items_w, int n_w, const double* wsd,
                                  char* ws, cudaStream_t st);
// The bounded-wait timeout path on purpose (a wait of `limit` tries, <= the kernels' own
// limit, on an mbarrier nothing arrives on): sets the status word's timeout bit.
cudaError_t launch_wait_selftest(unsigned* status, unsigned long long limit, cudaStream_t st);
// segments: some A operands carry one exponent per segment (a_nseg may exceed 1); otherwise
// every problem has a_nseg = 1.  digits: the nd (4..6) of every problem of the launch.
cudaError_t launch_split_gemm(const SplitGemmDesc* probs, const WorkItem* items, int nitems, const char* ws,
                              double* cbase, unsigned* status, cudaStream_t st, bool segments, int digits);

}  // namespace lx
