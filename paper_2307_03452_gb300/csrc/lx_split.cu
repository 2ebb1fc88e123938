// Split-precision transforms: the two GEMMs of the paper's Eq. make-abq and Eq. make-abcd
// evaluated as Ozaki-style sums of BF16 slice products on the tcgen05 tensor cores.
//
// Each FP64 operand row x is written as x = 2^(e - W) * q with a per-row power of two 2^e
// (|x| < 2^e over the row), q an integer of W = NSLICE * BETA bits, and q split into NSLICE
// balanced signed digits of BETA bits, q = sum_s d_s 2^(BETA (NSLICE-1-s)).  Every digit is
// an integer of magnitude <= 2^BETA, exact in BF16.  The product of two such rows is
//   sum_{s,t} 2^(BETA (2 NSLICE - 2 - s - t)) sum_k dA_s dB_t.
// Products with s + t <= NSLICE - 1 are kept; each diagonal d = s + t has its own TMEM
// accumulator, drained into 64-bit integers every SPLIT_SEG_KB K blocks so that every FP32
// partial sum stays an integer of magnitude <= 2^24 (exact), and the 64-bit sum is converted
// to FP64 once (the lowest BETA bits of the last diagonal are rounded off to keep the sum
// clear of 64-bit overflow).  FP64 arithmetic, which is scarce on this GPU, is used for none
// of it: the splitting works on the bit patterns of the FP64 inputs.
//
// Kernels:
//   split_operands_kernel  rows q of the [p|q] operand gathered from [r]^(0), and the H
//                      rows, -> digit planes + row exponents (GEMM1 operands, H_ket)
//   split_rows_kernel  FP64 row-major matrix rows ([ab|q]) -> digit planes + row exponents
//   split_gemm_kernel  D = A B^T on tcgen05 (M tile 128, N tile <= 32, K blocks of 32),
//                      persistent, operand blocks streamed by bulk TMA copies into a
//                      3-stage mbarrier ring, one thread issuing the MMAs, two TMEM
//                      accumulator sets drained by eight warps.
#include <cstdint>
#include <mutex>
#include <vector>

#include "lx_internal.cuh"
#include "lx_split.cuh"

namespace lx {

namespace {

constexpr unsigned long long WAIT_LIMIT = 1ull << 24;  // bounded spin: then flag and bail out


__device__ inline void set_status(unsigned* st, unsigned bit) { atomicOr(st, bit); }

__device__ inline uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ inline void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ inline void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ inline bool mbar_try_wait(uint64_t* bar, uint32_t phase) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(phase)
        : "memory");
    return ok != 0;
}

// Bounded wait on an mbarrier phase; false (and the status bit) when `limit` tries are spent.
__device__ inline bool mbar_wait(uint64_t* bar, uint32_t phase, unsigned* status,
                                 unsigned long long limit = WAIT_LIMIT) {
    for (unsigned long long i = 0; i < limit; ++i)
        if (mbar_try_wait(bar, phase)) return true;
    set_status(status, ST_TIMEOUT);
    return false;
}

// The timeout path of the bounded waits, on purpose: one thread waits, with `limit` tries,
// on an mbarrier that nothing arrives on (no copy is in flight, no TMEM is held), sets the
// status bit and returns.
__global__ void wait_selftest_kernel(unsigned* status, unsigned long long limit) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x != 0) return;
    mbar_init(&bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    mbar_wait(&bar, 0, status, limit);
}

// Bulk (non-tensor) TMA copy global -> shared; completes `bytes` of transaction on `bar`.
__device__ inline void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

__device__ inline void tmem_alloc(uint32_t* dst, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst)),
                 "r"(ncols)
                 : "memory");
}
__device__ inline void tmem_relinquish() {
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ inline void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ inline void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ inline void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Shared-memory matrix descriptor, K-major, no swizzle: core matrices of 8 rows x 16 bytes;
// lbo = byte distance between core matrices adjacent in K, sbo = adjacent in M/N.
__device__ inline uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFF);
    d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;  // descriptor version for tcgen05
    return d;                // base offset 0, no swizzle
}

// Instruction descriptor, kind::f16: BF16 x BF16 -> FP32, both operands K-major.
__device__ inline uint32_t idesc_bf16(int M, int N) {
    return (1u << 4)                    // D format: F32
           | (1u << 7)                  // A format: BF16
           | (1u << 10)                 // B format: BF16
           | ((uint32_t)(N >> 3) << 17)  // N / 8
           | ((uint32_t)(M >> 4) << 24); // M / 16
}

__device__ inline void umma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc)
        : "memory");
}

__device__ inline void umma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

__device__ inline void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
}
__device__ inline void tmem_ld8(uint32_t taddr, uint32_t (&r)[8]) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr)
                 : "memory");
}
__device__ inline void tmem_ld_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// ------------------------------------------------------------------ splitting

// Biased exponent field of an FP64 value (0 for zero / subnormal).
__device__ inline int exp_field(double x) { return (int)((__double_as_longlong(x) >> 52) & 0x7FF); }

// x * 2^s by exponent arithmetic (exact; underflow to zero).
__device__ inline double scale2(double x, int s) {
    const long long bits = __double_as_longlong(x);
    const int ex = (int)((bits >> 52) & 0x7FF);
    if (ex == 0 || s == 0) return ex == 0 ? 0.0 : x;
    const int ne = ex + s;
    if (ne <= 0) return 0.0;
    if (ne >= 2047) return __longlong_as_double((bits & (1ll << 63)) | 0x7FF0000000000000ll);
    return __longlong_as_double((bits & ~(0x7FFll << 52)) | ((long long)ne << 52));
}

// Biased exponent field of x 2^s: 0 if x is zero or subnormal or x 2^s underflows the normal
// range (the value scale2 would give), capped at 2047.
__device__ inline int exp_field_scaled(double x, int s) {
    const int ex = exp_field(x);
    return ex > 0 ? min(max(ex + s, 0), 2047) : 0;
}

// q = round(x 2^s 2^(W - e)) for |x 2^s| < 2^e, from the bit pattern (no FP64 arithmetic);
// equal to the rounding of scale2(x, s), so a scaled value that underflows gives 0.
__device__ inline long long fixed_of(double x, int s, int e) {
    const long long bits = __double_as_longlong(x);
    const int ex = (int)((bits >> 52) & 0x7FF);
    const int ne = ex + s;
    if (ex == 0 || ne <= 0) return 0;  // zero or subnormal: below any row scale that matters
    const long long mant = (bits & 0xFFFFFFFFFFFFFll) | (1ll << 52);
    const int rs = 1075 - ne - SPLIT_W + e;  // right shift, >= 53 - W > 0
    long long q = 0;
    if (rs < 63) q = (mant + (1ll << (rs - 1))) >> rs;
    return bits < 0 ? -q : q;
}

// The digits of q (|q| <= 2^48), most significant first, balanced: |d_0| <= 2^BETA and
// -2^(BETA-1) <= d_s < 2^(BETA-1) for s > 0.  Adding B = 2^(BETA-1) (1 + 256 + ... + 256^4)
// makes the five low digits plain bytes: byte j of y = q + B is d_(5-j) + 128, with every
// carry done by the one 64-bit add, and d_0 = floor(y / 2^40).  Each byte becomes an FP32 bit
// pattern with one byte permute: [byte, 0, 0x40, 0x4B] is the FP32 number 1.5 2^23 + byte,
// so subtracting 1.5 2^23 + 128 leaves d exactly.  A digit has at most 8 significant bits,
// so its BF16 pattern is the upper half of its FP32 pattern.
static_assert(SPLIT_NSLICE == 6 && SPLIT_BETA == 8, "digit extraction assumes 6 digits of 8 bits");
__device__ inline void digits_of(long long q, uint32_t (&f)[SPLIT_NSLICE]) {
    const long long y = q + 0x8080808080ll;
    const uint32_t lo = (uint32_t)y;
    const int hi = (int)(y >> 32);
    constexpr uint32_t MAGIC = 0x4B400000u;  // 1.5 2^23
    constexpr float BIAS = 12582912.0f + 128.0f;
    f[5] = __float_as_uint(__uint_as_float(__byte_perm(lo, MAGIC, 0x7650)) - BIAS);
    f[4] = __float_as_uint(__uint_as_float(__byte_perm(lo, MAGIC, 0x7651)) - BIAS);
    f[3] = __float_as_uint(__uint_as_float(__byte_perm(lo, MAGIC, 0x7652)) - BIAS);
    f[2] = __float_as_uint(__uint_as_float(__byte_perm(lo, MAGIC, 0x7653)) - BIAS);
    f[1] = __float_as_uint(__uint_as_float(__byte_perm((uint32_t)hi, MAGIC, 0x7650)) - BIAS);
    f[0] = __float_as_uint(__int_as_float((int)MAGIC + (hi >> 8)) - 12582912.0f);
}

// Digits of 8 consecutive values (k0 .. k0+7, k0 a multiple of 8) of one row, written as one
// 16-byte store per slice (one row of a core matrix), for the first nd slices.
__device__ inline int64_t dig_index(int row, int k, int s, int T, int nkb);
__device__ inline void store_digit_group(__nv_bfloat16* dig, int row, int k0, int T, int nkb,
                                         const long long (&q)[8], int nd) {
    // w[s][i]: BF16 pair of slice s, element 2i in the low half and 2i + 1 in the high half
    uint32_t w[SPLIT_NSLICE][4];
#pragma unroll
    for (int j = 0; j < 8; j += 2) {
        uint32_t f0[SPLIT_NSLICE], f1[SPLIT_NSLICE];
        digits_of(q[j], f0);
        digits_of(q[j + 1], f1);
#pragma unroll
        for (int s = 0; s < SPLIT_NSLICE; ++s) w[s][j >> 1] = __byte_perm(f0[s], f1[s], 0x7632);
    }
#pragma unroll
    for (int s = 0; s < SPLIT_NSLICE; ++s)  // slices past nd are never read
        if (s < nd)
            *reinterpret_cast<uint4*>(dig + dig_index(row, k0, s, T, nkb)) =
                make_uint4(w[s][0], w[s][1], w[s][2], w[s][3]);
}

// Offset (in BF16 elements) of element (row, k) of slice s inside an operand stored as
// row tiles of T rows and K blocks of SPLIT_KB: block (rt, kb) holds NSLICE slice-blocks of
// T x KB elements, each in core matrices (8 rows x 8 elements) ordered (row/8, k/8).
__device__ inline int64_t dig_index(int row, int k, int s, int T, int nkb) {
    const int rt = row / T, r = row - rt * T, kb = k / SPLIT_KB, kk = k - kb * SPLIT_KB;
    const int64_t block = ((int64_t)rt * nkb + kb) * SPLIT_NSLICE + s;
    return block * (T * SPLIT_KB) + ((r >> 3) * (SPLIT_KB / 8) + (kk >> 3)) * 64 + (r & 7) * 8 + (kk & 7);
}

// split_rows_kernel gives one warp 8 consecutive rows r0 .. r0+7 (r0 a multiple of 8), taken
// as four pairs.  For a pair, lane (rr, c) = (lane / 16, lane % 16) handles row r0 + 2i + rr and
// the 8-column groups c, c + 16, c + 32, ... (columns 128 j + 8c .. 128 j + 8c + 7).  A pair is
// read twice, once for its exponent and once for its digits; the two reads are close enough
// in time that the second comes from L1 or L2.  The two rows of a pair are adjacent in every
// core matrix, so each 32-byte sector of the digit planes is written whole.

// Largest exponent field over the 16 lanes of a row.
__device__ inline int row_max16(int mx) {
#pragma unroll
    for (int o = 8; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    return mx;
}

// Split 8 rows (4 pairs) through value(row, k0, v[8], sh[8]) (values and the powers of two
// they are scaled by; zeros outside the matrix): digit planes of row tile T with nkb K blocks
// and one int exponent per row (the modes of SplitRowsDesc::fixed).
template <bool SEGMENTS, typename Value>
__device__ __forceinline__ void split_8rows(int r0, int nkb, int T, int fixed, int nseg, int nd,
                                            __nv_bfloat16* __restrict__ dig, int* __restrict__ exps, Value value) {
    const int lane = threadIdx.x & 31, c8 = 8 * (lane & 15);
    static_assert(SPLIT_SEG_KB * SPLIT_KB == 128, "one pass of a row pair covers one segment");
    for (int pr = 0; pr < 4; ++pr) {
        const int row = r0 + 2 * pr + (lane >> 4);
        if (SEGMENTS && fixed == 2) {
            // one exponent per segment of 128 columns: one pass of the row's 16 lanes covers a
            // segment (every lane takes every pass, for the shuffles; columns past the K blocks
            // read as zeros and are not stored)
            for (int sg = 0; sg < nseg; ++sg) {
                const int k0 = 128 * sg + c8;
                double v[8];
                int sh[8];
                value(row, k0, v, sh);
                int mx = 0;
#pragma unroll
                for (int i = 0; i < 8; ++i) mx = max(mx, exp_field_scaled(v[i], sh[i]));
                mx = row_max16(mx);
                const int e = mx > 0 ? mx - 1022 : SPLIT_EXP_NONE;
                if (k0 < nkb * SPLIT_KB) {
                    long long q[8];
#pragma unroll
                    for (int i = 0; i < 8; ++i) q[i] = mx > 0 ? fixed_of(v[i], sh[i], e) : 0ll;
                    store_digit_group(dig, row, k0, T, nkb, q, nd);
                }
                if ((lane & 15) == 0) exps[(int64_t)row * nseg + sg] = e;
            }
            continue;
        }
        int mx = fixed == 1 ? 1022 : 0;  // 1022: the exponent field bound of values in (-1, 1)
        if (fixed == 0) {
            for (int k0 = c8; k0 < nkb * SPLIT_KB; k0 += 128) {
                double v[8];
                int sh[8];
                value(row, k0, v, sh);
#pragma unroll
                for (int i = 0; i < 8; ++i) mx = max(mx, exp_field_scaled(v[i], sh[i]));
            }
            mx = row_max16(mx);
        }
        const int e = mx > 0 ? mx - 1022 : 0;  // |x| < 2^e over the row
        for (int k0 = c8; k0 < nkb * SPLIT_KB; k0 += 128) {
            double v[8];
            int sh[8];
            value(row, k0, v, sh);
            long long q[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) q[i] = mx > 0 ? fixed_of(v[i], sh[i], e) : 0ll;
            store_digit_group(dig, row, k0, T, nkb, q, nd);
        }
        if ((lane & 15) == 0) exps[row] = e;
    }
}

// One split_rows item (item.q = descriptor, item.a = r0), by one warp (SEGMENTS: fixed = 2 may
// occur).
template <bool SEGMENTS>
__device__ __forceinline__ void split_rows_item(const SplitRowsDesc* __restrict__ descs, const WorkItem& it,
                                                const double* __restrict__ src_base, char* __restrict__ ws) {
    const SplitRowsDesc d = descs[it.q];
    const double* src = src_base + d.src_off;
    const int* shift = d.shift_off >= 0 ? reinterpret_cast<const int*>(ws + d.shift_off) : nullptr;
    split_8rows<SEGMENTS>(it.a, d.nkb, d.T, d.fixed, d.nseg, d.nd, reinterpret_cast<__nv_bfloat16*>(ws + d.dig_off),
                reinterpret_cast<int*>(ws + d.exp_off), [&](int row, int k0, double (&v)[8], int (&sh)[8]) {
                    const bool live = row < d.rows;
                    const double* sr = src + (int64_t)row * d.ld;
#pragma unroll
                    for (int i = 0; i < 8; ++i) {
                        const int k = k0 + i;
                        const bool in = live && k < d.K;
                        v[i] = in ? sr[k] : 0.0;
                        sh[i] = in && shift ? d.shift_sign * shift[k] : 0;
                    }
                });
}

__global__ void __launch_bounds__(256) split_rows_kernel(const SplitRowsDesc* __restrict__ descs,
                                                         const WorkItem* __restrict__ items, int nitems,
                                                         const double* __restrict__ src_base, char* __restrict__ ws) {
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (warp >= nitems) return;
    split_rows_item<true>(descs, items[warp], src_base, ws);
}

// Rows q of the GEMM1 A operand: A[q][k] = [p+q]^(0) of primitive quartet (kp, kq) with
// k = kp*Np + p, q = kq*Nq + qq, scaled by 2^c1[k].  item.q = quartet, item.a = r0.  Here
// the 8 rows are processed at once: lane (rr, c) = (lane / 4, lane % 4) handles row r0 + rr
// and columns 8c .. 8c+7 of every K block, so the gathers of neighbouring rows (neighbouring
// Hermite indices) fall close together; the rows are gathered twice, once for the exponent.
// The position of [p+q]^(0) in [r]^(0) comes from the class's index table (gidx_offset): 8
// consecutive p of one primitive pair are one 16-byte load when they start on a multiple of 8
// within the pair's block, which every group does when K_bra = 1.
__device__ const uint16_t* g_gidx;

// One split_r item (item.q = quartet, item.a = r0), by one warp.
__device__ __forceinline__ void split_r_item(const DQuartet* __restrict__ qd, const SplitQuartet* __restrict__ sq,
                                             const WorkItem& it, const double* __restrict__ wsd,
                                             char* __restrict__ ws) {
    const int lane = threadIdx.x & 31;
    const DQuartet q = qd[it.q];
    const SplitQuartet s = sq[it.q];
    const int row = it.a + (lane >> 2), c8 = 8 * (lane & 3);
    const int nrow = q.kket * q.nq, K = q.kbra * q.np;
    const bool live = row < nrow;
    const int kq = live ? row / q.nq : 0;
    const double* Rr = wsd + q.rr_off + (int64_t)kq * q.nr;
    const int64_t kp_stride = (int64_t)q.kket * q.nr;
    const int* c1 = reinterpret_cast<const int*>(ws + s.c1_off);
    // this row's positions hidx(p + q) for p < Np
    const uint16_t* G = g_gidx + s.gidx_off + (int64_t)(row - kq * q.nq) * ((q.np + 7) / 8 * 8);
    // [p+q]^(0) of columns k0 .. k0+7 (unscaled) and their shifts, walking (kp, p)
    auto group = [&](int k0, double (&v)[8], int (&sh)[8]) {
        int kp = k0 / q.np, p = k0 - kp * q.np;
        if (live && (p & 7) == 0 && p + 8 <= q.np && k0 + 8 <= K) {
            // one primitive pair, 16-byte aligned: vector loads of positions and shifts
            const uint4 g = *reinterpret_cast<const uint4*>(G + p);
            const int4 ca = *reinterpret_cast<const int4*>(c1 + k0);
            const int4 cb = *reinterpret_cast<const int4*>(c1 + k0 + 4);
            const double* Rk = Rr + kp * kp_stride;
            v[0] = Rk[g.x & 0xFFFF], v[1] = Rk[g.x >> 16], v[2] = Rk[g.y & 0xFFFF], v[3] = Rk[g.y >> 16];
            v[4] = Rk[g.z & 0xFFFF], v[5] = Rk[g.z >> 16], v[6] = Rk[g.w & 0xFFFF], v[7] = Rk[g.w >> 16];
            sh[0] = ca.x, sh[1] = ca.y, sh[2] = ca.z, sh[3] = ca.w;
            sh[4] = cb.x, sh[5] = cb.y, sh[6] = cb.z, sh[7] = cb.w;
            return;
        }
        int k = k0;
#pragma unroll
        for (int i = 0; i < 8; ++i, ++k) {
            double x = 0.0;
            int h = 0;
            if (live && k < K) {
                x = Rr[kp * kp_stride + G[p]];
                h = c1[k];
            }
            v[i] = x;
            sh[i] = h;
            if (++p == q.np) {
                p = 0;
                ++kp;
            }
        }
    };
    // exponent pass: the exponent field of x 2^c1 is that of x plus c1 (zeros stay zero)
    int mx = 0;
    for (int kb = 0; kb < s.nkb1; ++kb) {
        double v[8];
        int sh[8];
        group(SPLIT_KB * kb + c8, v, sh);
#pragma unroll
        for (int i = 0; i < 8; ++i) mx = max(mx, exp_field_scaled(v[i], sh[i]));
    }
    mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, 1));
    mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, 2));
    const int e = mx > 0 ? mx - 1022 : 0;
    __nv_bfloat16* dig = reinterpret_cast<__nv_bfloat16*>(ws + s.a1_dig);
    for (int kb = 0; kb < s.nkb1; ++kb) {
        double v[8];
        int sh[8];
        group(SPLIT_KB * kb + c8, v, sh);
        long long qv[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) qv[i] = mx > 0 ? fixed_of(v[i], sh[i], e) : 0ll;
        store_digit_group(dig, row, SPLIT_KB * kb + c8, SPLIT_TA, s.nkb1, qv, s.nd);
    }
    if ((lane & 3) == 0) reinterpret_cast<int*>(ws + s.a1_exp)[row] = e;
}

// The operands of GEMM1 and the H operand of GEMM2 in one launch: split_r items ([p|q]^T rows,
// issue-bound gathers) and split_rows items (H rows, load-latency bound) in alternating blocks,
// so that the two kinds share the SMs.  8 warps (items) per block.
__global__ void __launch_bounds__(256) split_operands_kernel(const DQuartet* __restrict__ qd,
                                                             const SplitQuartet* __restrict__ sq,
                                                             const WorkItem* __restrict__ items_r, int n_r,
                                                             const SplitRowsDesc* __restrict__ descs,
                                                             const WorkItem* __restrict__ items_w, int n_w,
                                                             const double* __restrict__ wsd, char* __restrict__ ws) {
    const int nb_r = (n_r + 7) / 8, nb_w = (n_w + 7) / 8, m = min(nb_r, nb_w);
    const int b = blockIdx.x;
    int kind, idx;  // kind 0: split_r, 1: split_rows
    if (b < 2 * m) {
        kind = b & 1;
        idx = b >> 1;
    } else {
        kind = nb_r > nb_w ? 0 : 1;
        idx = m + (b - 2 * m);
    }
    const int w = idx * 8 + (threadIdx.x >> 5);
    if (kind == 0) {
        if (w < n_r) split_r_item(qd, sq, items_r[w], wsd, ws);
    } else {
        if (w < n_w) split_rows_item<false>(descs, items_w[w], wsd, ws);  // H rows: fixed = 1
    }
}

// ------------------------------------------------------------------ tcgen05 GEMM

constexpr int STAGES = 3;
constexpr int NBUF = 2;  // TMEM accumulator sets: one drains while the other accumulates
constexpr int A_BLOCK = SPLIT_NSLICE * SPLIT_TA * SPLIT_KB * 2;  // bytes of one A block (all slices)
constexpr int B_BLOCK_MAX = SPLIT_NSLICE * SPLIT_TB * SPLIT_KB * 2;
constexpr int A_SLICE = SPLIT_TA * SPLIT_KB * 2;
constexpr int STAGE_BYTES = A_BLOCK + B_BLOCK_MAX;
constexpr int BUF_COLS = SPLIT_NSLICE * SPLIT_TB;  // TMEM columns of one accumulator set
constexpr uint32_t TMEM_COLS = 512;
static_assert(NBUF * BUF_COLS <= (int)TMEM_COLS, "accumulator sets exceed TMEM");
constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 1024;
// warp 0 TMA, warp 1 MMA issue + TMEM, warps 2..9 drain / epilogue: two warps per TMEM lane
// quarter, each owning 16 of the tile's (at most 32) columns
constexpr int DRAIN_WARPS = 8;
constexpr int DCOLS = 16;  // columns per drain warp
constexpr int GEMM_THREADS = 32 * (2 + DRAIN_WARPS);
static_assert(SPLIT_TB == DCOLS * (DRAIN_WARPS / 4), "the drain warps cover the widest column tile");

__device__ inline void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// x / 2^s rounded to nearest (ties up), for s >= 0; 0 once the shift passes every bit.
__device__ inline long long shr_round(long long x, int s) {
    if (s <= 0) return x;
    if (s >= 62) return 0;
    return (x + (1ll << (s - 1))) >> s;
}

// Persistent: CTA b takes work items b, b + gridDim.x, ... (item.q = problem, item.a = M tile,
// item.b = N tile); the three roles walk the same sequence.  The TMA ring of K blocks runs
// on across item boundaries, and so do the two TMEM accumulator sets, so one tile's drains
// and output overlap the next tile's MMAs.
//
// Accumulation is exact.  Every digit is an integer with |d_0| <= 2^BETA and |d_s| <= 2^(BETA-1)
// for s > 0, so one k adds at most 2^17 to any diagonal d = s + t (2 * 2^15 + (d - 1) * 2^14 for
// d >= 2, 2^16 for d < 2).  The MMAs of SPLIT_SEG_KB K blocks (128 k) therefore leave every
// FP32 accumulator, and every partial sum on the way, an integer of magnitude <= 2^24, which
// FP32 holds exactly; the four drain warps then move the diagonals into 64-bit integers while
// the next segment accumulates in the other TMEM set.  Per k the combined value is at most
// 2^(2W - 48) = 2^48, so the 64-bit sum is shifted down by xs bits when K exceeds 2^14.
//
// The MMAs of one A slice s and one K step are issued against the B slices 0..nd-1-s at once:
// slice t lies tb rows after slice t-1 in shared memory and diagonal s + t lies tb TMEM
// columns after s + t - 1, so A_s [B_0; B_1; ...] lands every product on its diagonal in one
// MMA of N = (nd - s) tb <= 192.  With nd < NSLICE digits only the first nd slices of each
// operand block are loaded, nd MMAs are issued per K step and nd diagonals drained.
template <bool SEGS, int ND>
__global__ void __launch_bounds__(GEMM_THREADS, 1)
    split_gemm_kernel(const SplitGemmDesc* __restrict__ probs, const WorkItem* __restrict__ items, int nitems,
                      const char* __restrict__ ws, double* __restrict__ cbase, unsigned* status) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    // 1024-byte aligned operand stages
    unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    __shared__ __align__(8) uint64_t full_bar[STAGES], empty_bar[STAGES], seg_full[NBUF], seg_empty[NBUF], final_bar;
    __shared__ uint32_t tmem_base_sh;
    __shared__ int abort_sh;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (warp == 1) {
        tmem_alloc(&tmem_base_sh, TMEM_COLS);
        tmem_relinquish();
    }
    if (tid == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&full_bar[s], 1);
            mbar_init(&empty_bar[s], 1);
        }
        for (int b = 0; b < NBUF; ++b) {
            mbar_init(&seg_full[b], 1);
            mbar_init(&seg_empty[b], DRAIN_WARPS);
        }
        mbar_init(&final_bar, 1);
        abort_sh = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base_sh;

    if (warp == 0) {
        if (lane == 0) {
            // producer: stream the A and B blocks of every K block of every item into the ring
            int g = 0;  // K blocks issued so far
            bool ok = true;
            for (int w = blockIdx.x; w < nitems && ok; w += gridDim.x) {
                const WorkItem it = items[w];
                const SplitGemmDesc P = probs[it.q];
                const int b_block = SPLIT_NSLICE * P.tb * SPLIT_KB * 2;
                const char* a_src = ws + P.a_dig + (int64_t)it.a * P.nkb * A_BLOCK;
                const char* b_src = ws + P.b_dig + (int64_t)it.b * P.nkb * b_block;
                // rows of this A tile that exist (up to M rounded up to 8): a partial last tile
                // is copied slice by slice, its first vr rows only; the rows past them hold
                // whatever the stage held before and only reach output rows >= M, which the
                // drain discards
                const int vr = min(SPLIT_TA, ((P.M + 7) & ~7) - it.a * SPLIT_TA);
                // the first nd digit slices of each block (slices are the outer index of a block)
                constexpr int nd = ND;  // P.nd equals ND (the launch is chosen by it)
                const int a_bytes = nd * vr * SPLIT_KB * 2, b_bytes = nd * P.tb * SPLIT_KB * 2;
                for (int kb = 0; kb < P.nkb; ++kb, ++g) {
                    const int st = g % STAGES, use = g / STAGES;
                    if ((use > 0 && !mbar_wait(&empty_bar[st], (use - 1) & 1, status)) || *(volatile int*)&abort_sh) {
                        abort_sh = 1;
                        ok = false;
                        break;
                    }
                    unsigned char* sa = smem + st * STAGE_BYTES;
                    mbar_expect_tx(&full_bar[st], a_bytes + b_bytes);
                    if (vr == SPLIT_TA) {
                        bulk_g2s(sa, a_src + (int64_t)kb * A_BLOCK, a_bytes, &full_bar[st]);
                    } else {
                        for (int sl = 0; sl < nd; ++sl)
                            bulk_g2s(sa + sl * A_SLICE, a_src + (int64_t)kb * A_BLOCK + sl * A_SLICE,
                                     vr * SPLIT_KB * 2, &full_bar[st]);
                    }
                    bulk_g2s(sa + A_BLOCK, b_src + (int64_t)kb * b_block, b_bytes, &full_bar[st]);
                }
            }
            // no copy may still be landing in shared memory when the CTA exits
            for (int st = 0; st < STAGES && st < g; ++st) {
                const int last = g - 1 - ((g - 1 - st) % STAGES);
                if (!mbar_wait(&full_bar[st], (last / STAGES) & 1, status)) abort_sh = 1;
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // Descriptors are built once: the start-address field (bits 0-13, address / 16)
            // of a descriptor is advanced by adding offset / 16, which cannot carry out of
            // the field since shared memory ends below 2^18 bytes.
            const uint32_t sbase = smem_u32(smem);
            const uint64_t a_desc0 = smem_desc(sbase, 128, (SPLIT_KB / 8) * 128);
            const uint64_t b_desc0 = smem_desc(sbase + A_BLOCK, 128, (SPLIT_KB / 8) * 128);
            int g = 0, sgc = 0;  // K blocks consumed, segments issued
            bool ok = true;
            for (int w = blockIdx.x; w < nitems && ok; w += gridDim.x) {
                const WorkItem it = items[w];
                const SplitGemmDesc P = probs[it.q];
                const int tb = P.tb, nkb = P.nkb;
                constexpr int nd = ND;
                uint32_t idesc[ND];
#pragma unroll
                for (int s = 0; s < ND; ++s) idesc[s] = idesc_bf16(SPLIT_TA, (ND - s) * tb);
                for (int kb0 = 0; kb0 < nkb && ok; kb0 += SPLIT_SEG_KB, ++sgc) {
                    const int buf = sgc & 1, ub = sgc >> 1;
                    if (ub > 0) {
                        if (!mbar_wait(&seg_empty[buf], (ub - 1) & 1, status)) ok = false;
                        tc_fence_after();
                    }
                    if (!ok || *(volatile int*)&abort_sh) {
                        ok = false;
                        break;
                    }
                    const uint32_t dcol = tmem + buf * BUF_COLS;
                    const int kb1 = min(nkb, kb0 + SPLIT_SEG_KB);
                    for (int kb = kb0; kb < kb1; ++kb, ++g) {
                        const int st = g % STAGES;
                        if (!mbar_wait(&full_bar[st], (g / STAGES) & 1, status)) {
                            ok = false;
                            break;
                        }
                        tc_fence_after();
                        const uint64_t st_off = (uint64_t)((st * STAGE_BYTES) >> 4);
                        const uint64_t ad0 = a_desc0 + st_off, bd0 = b_desc0 + st_off;
#pragma unroll
                        for (int ks = 0; ks < SPLIT_KB / 16; ++ks) {
#pragma unroll
                            for (int s = 0; s < ND; ++s) {
                                // the slice-0 MMA of a segment's first K step covers every diagonal
                                const uint32_t acc = (ks == 0 && s == 0 && kb == kb0) ? 0u : 1u;
                                umma_bf16(dcol + s * tb, ad0 + ((s * A_SLICE + ks * 256) >> 4), bd0 + ((ks * 256) >> 4),
                                          idesc[s], acc);
                            }
                        }
                        umma_commit(&empty_bar[st]);  // the stage is free once these MMAs have read it
                    }
                    if (!ok) break;
                    umma_commit(&seg_full[buf]);
                }
            }
            if (!ok) abort_sh = 1;
            // every MMA issued has completed before TMEM is released
            umma_commit(&final_bar);
            if (!mbar_wait(&final_bar, 0, status)) abort_sh = 1;
        }
    } else {
        // drain / epilogue: warp w reads TMEM lanes (rows) 32 (w % 4) .. 32 (w % 4) + 31 and the
        // DCOLS columns c0 .. c0 + DCOLS - 1 of each diagonal
        const int quarter = warp & 3, c0 = DCOLS * ((warp - 2) >> 2);
        const uint32_t lane_base = tmem + ((uint32_t)(quarter * 32) << 16) + c0;
        int sgc = 0;
        bool ok = true;
        for (int w = blockIdx.x; w < nitems && ok; w += gridDim.x) {
            const WorkItem it = items[w];
            const SplitGemmDesc P = probs[it.q];
            const int tb = P.tb, nkb = P.nkb;
            constexpr int nd = ND;
            const int m0 = it.a * SPLIT_TA, n0 = it.b * tb;
            const int nt = min(tb, P.N - n0);
            const bool mine = c0 < nt;  // warp-uniform
            const int xs = max(0, 32 - __clz(nkb * SPLIT_KB - 1) - 14);  // ceil(log2 K) - 14, if positive
            const int row = m0 + quarter * 32 + lane;
            const bool rlive = row < P.M;  // rows past M may come from stale shared memory: dropped
            // SEGS (A exponents per segment): acc 2^E is the row's sum so far, E the largest
            // exponent of its segments so far; each segment's exponent is read one segment ahead.
            // Otherwise one exponent per row, read at the end.
            constexpr bool segs = SEGS;
            const int* a_exp = reinterpret_cast<const int*>(ws + P.a_exp) + (int64_t)row * P.a_nseg;
            int E = SPLIT_EXP_NONE, es_next = segs && rlive ? a_exp[0] : SPLIT_EXP_NONE;
            long long acc[DCOLS];
#pragma unroll
            for (int j = 0; j < DCOLS; ++j) acc[j] = 0;
            for (int kb0 = 0, sg = 0; kb0 < nkb; kb0 += SPLIT_SEG_KB, ++sg, ++sgc) {
                const int buf = sgc & 1;
                int sa = 0, sv = 0;  // right shifts of the running sum and of this segment
                if (segs) {
                    const int es = es_next;
                    if (kb0 + SPLIT_SEG_KB < nkb) es_next = rlive ? a_exp[sg + 1] : SPLIT_EXP_NONE;
                    if (es > E) {
                        sa = E == SPLIT_EXP_NONE ? 62 : es - E;
                        E = es;
                    } else {
                        sv = E - es;  // a zero segment (es = SPLIT_EXP_NONE) contributes nothing
                    }
                    // the running sum's shift is the same for every column: applied here, once
                    if (sa > 0) {
#pragma unroll
                        for (int j = 0; j < DCOLS; ++j) acc[j] = shr_round(acc[j], sa);
                    }
                }
                // this segment's shift and its rounding half (sv >= 62: nothing left of it)
                const bool seg_live = sv < 62;
                const long long seg_half = sv > 0 && seg_live ? (1ll << (sv - 1)) : 0ll;
                const bool got = mbar_wait(&seg_full[buf], (sgc >> 1) & 1, status);
                ok = __all_sync(0xffffffffu, got) && !*(volatile int*)&abort_sh;
                if (!ok) break;
                tc_fence_after();
                if (mine) {
                    // the nd diagonals of HC columns in flight before one wait (the aligned sum
                    // takes its 16 columns in two halves, to stay within the registers)
                    constexpr int HC = SEGS ? 8 : DCOLS;
#pragma unroll
                    for (int h = 0; h < DCOLS / HC; ++h) {
                        uint32_t r[ND][HC];
#pragma unroll
                        for (int dg = 0; dg < ND; ++dg) {
                            if constexpr (HC == 16)
                                tmem_ld16(lane_base + buf * BUF_COLS + dg * tb, r[dg]);
                            else
                                tmem_ld8(lane_base + buf * BUF_COLS + dg * tb + HC * h, r[dg]);
                        }
                        tmem_ld_wait();
                        // v = sum_d G_d 2^(BETA (nd-2-d)) (>> xs); the last diagonal is rounded down BETA bits
#pragma unroll
                        for (int jj = 0; jj < HC; ++jj) {
                            long long v = 0;
#pragma unroll
                            for (int dg = 0; dg < ND; ++dg) {
                                const long long gv = (long long)__float2int_rn(__uint_as_float(r[dg][jj]));
                                if (dg < nd - 1)
                                    v += gv << (SPLIT_BETA * (nd - 2 - dg));
                                else
                                    v += (gv + (1ll << (SPLIT_BETA - 1))) >> SPLIT_BETA;
                            }
                            if (xs) v = (v + (1ll << (xs - 1))) >> xs;
                            const int j = HC * h + jj;
                            if (segs) {
                                if (seg_live) acc[j] += (v + seg_half) >> sv;
                            } else {
                                acc[j] += v;
                            }
                        }
                    }
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&seg_empty[buf]);
            }
            if (!ok) break;
            if (mine && rlive) {
                const int ea = segs ? E : reinterpret_cast<const int*>(ws + P.a_exp)[row];
                const int* eb_tab = reinterpret_cast<const int*>(ws + P.b_exp);
#pragma unroll
                for (int j = 0; j < DCOLS; ++j) {
                    const int col = n0 + c0 + j;
                    if (c0 + j < nt) {
                        // D = 2^(eA + eB - BETA nd + xs) * acc: one rounding (int64 -> FP64, to
                        // nearest even), then an exact power-of-two scaling (acc = 0 gives 0)
                        const int scale = ea + eb_tab[col] - SPLIT_BETA * nd + xs;
                        const double v = scale2(__ll2double_rn(acc[j]), scale);
                        if (P.transpose)
                            cbase[P.c_off + (int64_t)col * P.ldc + row] = v;
                        else
                            cbase[P.c_off + (int64_t)row * P.ldc + col] = v;
                    }
                }
            }
        }
        if (!ok) abort_sh = 1;
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) tmem_dealloc(tmem, TMEM_COLS);
}

}  // namespace

cudaError_t launch_split_rows(const SplitRowsDesc* descs, const WorkItem* items, int nitems, const double* src_base,
                              char* ws, cudaStream_t st) {
    if (nitems <= 0) return cudaSuccess;
    const int warps_per_block = 8;
    split_rows_kernel<<<(nitems + warps_per_block - 1) / warps_per_block, 32 * warps_per_block, 0, st>>>(
        descs, items, nitems, src_base, ws);
    return cudaGetLastError();
}

cudaError_t launch_split_operands(const DQuartet* qd, const SplitQuartet* sq, const WorkItem* items_r, int n_r,
                                  const SplitRowsDesc* descs, const WorkItem* items_w, int n_w, const double* wsd,
                                  char* ws, cudaStream_t st) {
    const int nb = (n_r + 7) / 8 + (n_w + 7) / 8;
    if (nb <= 0) return cudaSuccess;
    split_operands_kernel<<<nb, 256, 0, st>>>(qd, sq, items_r, n_r, descs, items_w, n_w, wsd, ws);
    return cudaGetLastError();
}

cudaError_t init_split_kernels(const int* host_tuv) {
    cudaError_t e = cudaSuccess;
    // the [p+q] index table (built once per process; a device copy per device, kept for the
    // life of the process)
    static std::vector<uint16_t> table;
    static std::mutex table_mutex;
    {
        std::lock_guard<std::mutex> lock(table_mutex);
        if (table.empty()) {
            table.assign((size_t)gidx_offset(GIDX_L, 0), 0);
            for (int lb = 0; lb < GIDX_L; ++lb)
                for (int lk = 0; lk < GIDX_L; ++lk) {
                    uint16_t* blk = table.data() + gidx_offset(lb, lk);
                    for (int q = 0; q < pyr(lk); ++q)
                        for (int p = 0; p < pyr(lb); ++p) {
                            const int a = host_tuv[p], b = host_tuv[q];
                            const int t = (a & 255) + (b & 255), u = ((a >> 8) & 255) + ((b >> 8) & 255),
                                      v = (a >> 16) + (b >> 16);
                            blk[(size_t)q * gidx_ld(lb) + p] = (uint16_t)hidx(t, u, v);
                        }
                }
        }
    }
    void* dev_table = nullptr;
    if ((e = cudaMalloc(&dev_table, sizeof(uint16_t) * table.size())) != cudaSuccess) return e;
    if ((e = cudaMemcpy(dev_table, table.data(), sizeof(uint16_t) * table.size(), cudaMemcpyHostToDevice)) !=
        cudaSuccess)
        return e;
    const uint16_t* p = static_cast<const uint16_t*>(dev_table);
    if ((e = cudaMemcpyToSymbol(g_gidx, &p, sizeof(p))) != cudaSuccess) return e;
    const void* kernels[] = {(const void*)split_gemm_kernel<false, 4>, (const void*)split_gemm_kernel<false, 5>,
                             (const void*)split_gemm_kernel<false, 6>, (const void*)split_gemm_kernel<true, 4>,
                             (const void*)split_gemm_kernel<true, 5>,  (const void*)split_gemm_kernel<true, 6>};
    for (const void* k : kernels)
        if ((e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES)) != cudaSuccess)
            return e;
    return cudaSuccess;
}

cudaError_t launch_wait_selftest(unsigned* status, unsigned long long limit, cudaStream_t st) {
    if (limit > WAIT_LIMIT) return cudaErrorInvalidValue;
    wait_selftest_kernel<<<1, 32, 0, st>>>(status, limit);
    return cudaGetLastError();
}

cudaError_t launch_split_gemm(const SplitGemmDesc* probs, const WorkItem* items, int nitems, const char* ws,
                              double* cbase, unsigned* status, cudaStream_t st, bool segments, int digits) {
    if (nitems <= 0) return cudaSuccess;
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    // one CTA per SM (the TMEM allocation and the operand ring take the whole SM)
    const int grid = nitems < sms ? nitems : sms;
#define LX_SPLIT_GEMM(S, D) split_gemm_kernel<S, D><<<grid, GEMM_THREADS, SMEM_BYTES, st>>>(probs, items, nitems, ws, cbase, status)
    switch ((segments ? 8 : 0) + digits) {
        case 4: LX_SPLIT_GEMM(false, 4); break;
        case 5: LX_SPLIT_GEMM(false, 5); break;
        case 6: LX_SPLIT_GEMM(false, 6); break;
        case 12: LX_SPLIT_GEMM(true, 4); break;
        case 13: LX_SPLIT_GEMM(true, 5); break;
        case 14: LX_SPLIT_GEMM(true, 6); break;
        default: return cudaErrorInvalidValue;
    }
#undef LX_SPLIT_GEMM
    return cudaGetLastError();
}

}  // namespace lx
