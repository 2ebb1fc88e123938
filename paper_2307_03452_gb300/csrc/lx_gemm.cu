// The two Hermite-to-Cartesian/solid transforms as batched FP64 GEMMs (paper, Section 2:
// Eq. make-abq and Eq. make-abcd):
//   GEMM1  X[ab][kq*Nq + q] = sum_{kp, p} H_bra[ab][kp*Np + p] [p+q]^(0)_{kp,kq}
//          (the [p|q] operand is gathered on the fly from the [r]^(0) vector of each primitive
//          quartet; the (-1)^{l_q} of Eq. pq is carried by the ket H), bra primitives summed in
//          the reduction dimension.
//   GEMM2  out[ab][cd] = sum_{kq, q} X[ab][kq*Nq + q] H_ket[cd][kq*Nq + q], ket primitives
//          summed in the reduction dimension.
// FP64 on GB300 runs at one rate for DFMA and for the FP64 mma.sync; the tiles use
// mma.sync.m8n8k4.f64 so that the work is done in 8x8 blocks and ragged edges waste little.
// Each CTA (4 warps) owns a 32 x 64 output tile; 8x8 blocks wholly outside the matrix are skipped.
#include "lx_internal.cuh"

namespace lx {

namespace {

__device__ int g_tuv_gemm[NHERM_TOT];

constexpr int BM = GEMM_BM, BN = GEMM_BN, BK = GEMM_BK;
constexpr int APAD = 4, BPAD = 4;

__device__ __forceinline__ void dmma(double& c0, double& c1, double a, double b) {
    asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};\n"
                 : "+d"(c0), "+d"(c1)
                 : "d"(a), "d"(b));
}

template <int MODE>
__global__ void __launch_bounds__(128) gemm_kernel(const DQuartet* __restrict__ qd, const DPair* __restrict__ pairs,
                                                   const WorkItem* __restrict__ items,
                                                   const double* __restrict__ ws, double* __restrict__ cout) {
    __shared__ double As[BM][BK + APAD];
    __shared__ double Bs[BK][BN + BPAD];
    const WorkItem it = items[blockIdx.x];
    const DQuartet q = qd[it.q];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

    int M, N, K;
    const double* A;
    double* C;
    if (MODE == 1) {
        M = q.nab;
        N = q.kket * q.nq;
        K = q.kbra * q.np;
        A = ws + pairs[q.pb].h_off;
        C = cout + q.x_off;
    } else {
        M = q.nab;
        N = q.ncd;
        K = q.kket * q.nq;
        A = ws + q.x_off;
        C = cout + q.out_off;
    }
    const int lda = K, ldc = N;
    const int m0 = it.a * BM, n0 = it.b * BN;
    const int wm = (warp >> 1) * 16, wn = (warp & 1) * 32;

    // MODE 1: every thread gathers the same column n of the B tile across K steps.
    const int bn_col = tid & 63;
    int g_kq = 0, g_tq = 0;
    bool g_nvalid = false;
    const double* Rr = nullptr;
    if (MODE == 1) {
        const int n = n0 + bn_col;
        g_nvalid = n < N;
        if (g_nvalid) {
            g_kq = n / q.nq;
            g_tq = __ldg(&g_tuv_gemm[n - g_kq * q.nq]);
        }
        Rr = ws + q.rr_off;
    }
    const double* Bt = (MODE == 2) ? ws + pairs[q.pk].h_off : nullptr;

    double acc[2][4][2];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j][0] = acc[i][j][1] = 0.0;

    bool rowok[2], colok[4];
#pragma unroll
    for (int i = 0; i < 2; ++i) rowok[i] = m0 + wm + 8 * i < M;
#pragma unroll
    for (int j = 0; j < 4; ++j) colok[j] = n0 + wn + 8 * j < N;

    for (int k0 = 0; k0 < K; k0 += BK) {
        // A tile: 32 x 16, coalesced along k
#pragma unroll
        for (int e = tid; e < BM * BK; e += 128) {
            const int r = e >> 4, c = e & 15;
            const int m = m0 + r, k = k0 + c;
            As[r][c] = (m < M && k < K) ? A[(int64_t)m * lda + k] : 0.0;
        }
        if (MODE == 1) {
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int kk = (tid >> 6) + 2 * j;
                const int k = k0 + kk;
                double v = 0.0;
                if (g_nvalid && k < K) {
                    const int kp = k / q.np, p = k - kp * q.np;
                    const int tp = __ldg(&g_tuv_gemm[p]);
                    const int s = tp + g_tq;  // componentwise sum of packed (t, u, v)
                    const int r = hidx(s & 255, (s >> 8) & 255, s >> 16);
                    v = Rr[(int64_t)(kp * q.kket + g_kq) * q.nr + r];
                }
                Bs[kk][bn_col] = v;
            }
        } else {
#pragma unroll
            for (int e = tid; e < BK * BN; e += 128) {
                const int nn = e >> 4, kk = e & 15;
                const int n = n0 + nn, k = k0 + kk;
                Bs[kk][nn] = (n < N && k < K) ? Bt[(int64_t)n * K + k] : 0.0;
            }
        }
        __syncthreads();
#pragma unroll
        for (int ks = 0; ks < BK; ks += 4) {
            double af[2], bf[4];
#pragma unroll
            for (int i = 0; i < 2; ++i) af[i] = As[wm + 8 * i + (lane >> 2)][ks + (lane & 3)];
#pragma unroll
            for (int j = 0; j < 4; ++j) bf[j] = Bs[ks + (lane & 3)][wn + 8 * j + (lane >> 2)];
#pragma unroll
            for (int i = 0; i < 2; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    if (rowok[i] && colok[j]) dmma(acc[i][j][0], acc[i][j][1], af[i], bf[j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const int row = m0 + wm + 8 * i + (lane >> 2);
        if (row >= M) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int col = n0 + wn + 8 * j + 2 * (lane & 3);
            if (col < N) C[(int64_t)row * ldc + col] = acc[i][j][0];
            if (col + 1 < N) C[(int64_t)row * ldc + col + 1] = acc[i][j][1];
        }
    }
}

}  // namespace

cudaError_t init_tuv_table(const int* host_tuv) {
    return cudaMemcpyToSymbol(g_tuv_gemm, host_tuv, sizeof(int) * NHERM_TOT);
}

cudaError_t launch_gemm1(const DQuartet* qd, const DPair* pairs, const WorkItem* items, int nitems, double* ws,
                         unsigned* status, cudaStream_t st) {
    (void)status;
    if (nitems <= 0) return cudaSuccess;
    gemm_kernel<1><<<nitems, 128, 0, st>>>(qd, pairs, items, ws, ws);
    return cudaGetLastError();
}

cudaError_t launch_gemm2(const DQuartet* qd, const DPair* pairs, const WorkItem* items, int nitems,
                         const double* ws_in, double* out, unsigned* status, cudaStream_t st) {
    (void)status;
    if (nitems <= 0) return cudaSuccess;
    gemm_kernel<2><<<nitems, 128, 0, st>>>(qd, pairs, items, ws_in, out);
    return cudaGetLastError();
}

}  // namespace lx
