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
// Four tile shapes (32x64, 64x32, 32x32, 64x64 per CTA of 4 warps) exist; each work item
// names its shape (chosen by the planner from the autotuned table).  One persistent launch
// per shape in use walks all of that shape's items, so quartets of mixed classes and
// contraction degrees share a launch.  8x8 blocks wholly outside a ragged edge are skipped.
#include "lx_internal.cuh"

namespace lx {

namespace {

__device__ int g_tuv_gemm[NHERM_TOT];

constexpr int BK = GEMM_BK;
constexpr int PAD = 4;
constexpr int MAXBM = 64, MAXBN = 64;

__device__ __forceinline__ void dmma(double& c0, double& c1, double a, double b) {
    asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};\n"
                 : "+d"(c0), "+d"(c1)
                 : "d"(a), "d"(b));
}

struct GemmSmem {
    double As[MAXBM][BK + PAD];
    double Bs[BK][MAXBN + PAD];
};

// One output tile of one quartet; WM x WN blocks of 8x8 per warp, warps 2 x 2.
template <int MODE, int WM, int WN>
__device__ void gemm_tile(const DQuartet& q, const DPair* __restrict__ pairs, int mtile, int ntile,
                          const double* __restrict__ ws, double* __restrict__ cout, GemmSmem& sm) {
    constexpr int BM = 16 * WM, BN = 16 * WN;
    static_assert(128 % BN == 0, "each thread gathers one fixed column of the B tile");
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
    const int m0 = mtile * BM, n0 = ntile * BN;
    const int wm = (warp >> 1) * (8 * WM), wn = (warp & 1) * (8 * WN);

    const int bn_col = tid % BN, bk_row0 = tid / BN;
    constexpr int BK_STEP = 128 / BN;
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

    double acc[WM][WN][2];
#pragma unroll
    for (int i = 0; i < WM; ++i)
#pragma unroll
        for (int j = 0; j < WN; ++j) acc[i][j][0] = acc[i][j][1] = 0.0;
    // 8-row (8-column) blocks past the edge are skipped; a block holding exactly one row
    // (column) at the edge -- solid outputs have N_ab = (2l_a+1)(2l_b+1) = 1 mod 8 -- is done
    // with scalar FMAs over the 32 lanes (lane = column x k step) at 1/8 of the MMA's work,
    // in a loop of its own so that the MMA sequence stays as it is
    bool rowok[WM], colok[WN], row1[WM], col1[WN], mma_ok[WM][WN];
    bool edge = false;
#pragma unroll
    for (int i = 0; i < WM; ++i) {
        rowok[i] = m0 + wm + 8 * i < M;
        row1[i] = m0 + wm + 8 * i == M - 1;
    }
#pragma unroll
    for (int j = 0; j < WN; ++j) {
        colok[j] = n0 + wn + 8 * j < N;
        col1[j] = n0 + wn + 8 * j == N - 1;
    }
#pragma unroll
    for (int i = 0; i < WM; ++i)
#pragma unroll
        for (int j = 0; j < WN; ++j) {
            mma_ok[i][j] = rowok[i] && colok[j] && !row1[i] && !col1[j];
            edge |= rowok[i] && colok[j] && (row1[i] || col1[j]);
        }

    for (int k0 = 0; k0 < K; k0 += BK) {
        for (int e = tid; e < BM * BK; e += 128) {
            const int r = e / BK, c = e - r * BK;
            const int m = m0 + r, k = k0 + c;
            sm.As[r][c] = (m < M && k < K) ? A[(int64_t)m * lda + k] : 0.0;
        }
        if (MODE == 1) {
#pragma unroll
            for (int kk = bk_row0; kk < BK; kk += BK_STEP) {
                const int k = k0 + kk;
                double v = 0.0;
                if (g_nvalid && k < K) {
                    const int kp = k / q.np, p = k - kp * q.np;
                    const int tp = __ldg(&g_tuv_gemm[p]);
                    const int s = tp + g_tq;  // componentwise sum of packed (t, u, v)
                    const int r = hidx(s & 255, (s >> 8) & 255, s >> 16);
                    v = Rr[(int64_t)(kp * q.kket + g_kq) * q.nr + r];
                }
                sm.Bs[kk][bn_col] = v;
            }
        } else {
            for (int e = tid; e < BK * BN; e += 128) {
                const int nn = e / BK, kk = e - nn * BK;
                const int n = n0 + nn, k = k0 + kk;
                sm.Bs[kk][nn] = (n < N && k < K) ? Bt[(int64_t)n * K + k] : 0.0;
            }
        }
        __syncthreads();
#pragma unroll
        for (int ks = 0; ks < BK; ks += 4) {
            if (k0 + ks >= K) break;  // k steps wholly past K (zeros) are skipped
            double af[WM], bf[WN];
#pragma unroll
            for (int i = 0; i < WM; ++i) af[i] = sm.As[wm + 8 * i + (lane >> 2)][ks + (lane & 3)];
#pragma unroll
            for (int j = 0; j < WN; ++j) bf[j] = sm.Bs[ks + (lane & 3)][wn + 8 * j + (lane >> 2)];
#pragma unroll
            for (int i = 0; i < WM; ++i)
#pragma unroll
                for (int j = 0; j < WN; ++j)
                    if (mma_ok[i][j]) dmma(acc[i][j][0], acc[i][j][1], af[i], bf[j]);
        }
        if (edge) {
            // the one-row / one-column blocks: A[row][k lane%4] B[k lane%4][column lane/4]
            // (or A[row lane/4][k lane%4] B[k lane%4][column]) summed per lane over k
            for (int ks = 0; ks < BK && k0 + ks < K; ks += 4) {
#pragma unroll
                for (int i = 0; i < WM; ++i)
#pragma unroll
                    for (int j = 0; j < WN; ++j) {
                        if (!(rowok[i] && colok[j]) || !(row1[i] || col1[j])) continue;
                        const double a = sm.As[wm + 8 * i + (row1[i] ? 0 : lane >> 2)][ks + (lane & 3)];
                        const double b = sm.Bs[ks + (lane & 3)][wn + 8 * j + (row1[i] ? lane >> 2 : 0)];
                        acc[i][j][0] = fma(a, b, acc[i][j][0]);
                    }
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < WM; ++i)
#pragma unroll
        for (int j = 0; j < WN; ++j) {
            if (!(rowok[i] && colok[j])) continue;
            if (row1[i] || col1[j]) {
                // sum the four k partials (lanes 4c .. 4c+3); lane 4c then holds entry c
                double v = acc[i][j][0];
                v += __shfl_xor_sync(0xffffffffu, v, 1);
                v += __shfl_xor_sync(0xffffffffu, v, 2);
                if ((lane & 3) != 0) continue;
                const int row = m0 + wm + 8 * i + (row1[i] ? 0 : lane >> 2);
                const int col = n0 + wn + 8 * j + (row1[i] ? lane >> 2 : 0);
                if (row < M && col < N) C[(int64_t)row * ldc + col] = v;
                continue;
            }
            const int row = m0 + wm + 8 * i + (lane >> 2);
            if (row >= M) continue;
            const int col = n0 + wn + 8 * j + 2 * (lane & 3);
            if (col < N) C[(int64_t)row * ldc + col] = acc[i][j][0];
            if (col + 1 < N) C[(int64_t)row * ldc + col + 1] = acc[i][j][1];
        }
}

// Persistent, one instantiation per tile shape (each keeps its own register budget): every
// CTA takes the next item of its shape from a work counter (zero on entry) until none is
// left (item.q = quartet, item.a = M tile, item.b = N tile).  The planner groups items by
// shape and orders each group by decreasing cost.
template <int MODE, int WM, int WN>
__global__ void __launch_bounds__(128, WM * WN > 8 ? 4 : 8) gemm_kernel(const DQuartet* __restrict__ qd, const DPair* __restrict__ pairs,
                                                   const WorkItem* __restrict__ items, int nitems,
                                                   const double* __restrict__ ws, double* __restrict__ cout,
                                                   int* __restrict__ counter) {
    __shared__ GemmSmem sm;
    __shared__ int s_next;
    for (;;) {
        if (threadIdx.x == 0) s_next = atomicAdd(counter, 1);
        __syncthreads();
        const int w = s_next;
        __syncthreads();
        if (w >= nitems) break;
        const WorkItem it = items[w];
        const DQuartet q = qd[it.q];
        gemm_tile<MODE, WM, WN>(q, pairs, it.a, it.b, ws, cout, sm);
    }
}

int g_persist_grid[2][GEMM_NVARIANT];

template <int MODE, int WM, int WN>
cudaError_t occupancy(int sms, int& grid) {
    int b = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, gemm_kernel<MODE, WM, WN>, 128, 0);
    grid = sms * (b > 0 ? b : 1);
    return e;
}

template <int MODE>
cudaError_t launch_variants(const DQuartet* qd, const DPair* pairs, const WorkItem* items, const int* counts,
                            const double* ws, double* cout, int* counters, cudaStream_t st) {
    int off = 0;
    for (int v = 0; v < GEMM_NVARIANT; ++v) {
        const int n = counts[v];
        if (n <= 0) continue;
        const int cap = g_persist_grid[MODE - 1][v];
        const int grid = cap > 0 && n > cap ? cap : n;
        const WorkItem* it = items + off;
        switch (v) {
            case GEMM_V32x64: gemm_kernel<MODE, 2, 4><<<grid, 128, 0, st>>>(qd, pairs, it, n, ws, cout, counters + v); break;
            case GEMM_V64x32: gemm_kernel<MODE, 4, 2><<<grid, 128, 0, st>>>(qd, pairs, it, n, ws, cout, counters + v); break;
            case GEMM_V32x32: gemm_kernel<MODE, 2, 2><<<grid, 128, 0, st>>>(qd, pairs, it, n, ws, cout, counters + v); break;
            default: gemm_kernel<MODE, 4, 4><<<grid, 128, 0, st>>>(qd, pairs, it, n, ws, cout, counters + v); break;
        }
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        off += n;
    }
    return cudaSuccess;
}

}  // namespace

cudaError_t init_tuv_table(const int* host_tuv) {
    cudaError_t e = cudaMemcpyToSymbol(g_tuv_gemm, host_tuv, sizeof(int) * NHERM_TOT);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    int* g1 = g_persist_grid[0];
    int* g2 = g_persist_grid[1];
    if ((e = occupancy<1, 2, 4>(sms, g1[GEMM_V32x64])) != cudaSuccess ||
        (e = occupancy<1, 4, 2>(sms, g1[GEMM_V64x32])) != cudaSuccess ||
        (e = occupancy<1, 2, 2>(sms, g1[GEMM_V32x32])) != cudaSuccess ||
        (e = occupancy<1, 4, 4>(sms, g1[GEMM_V64x64])) != cudaSuccess ||
        (e = occupancy<2, 2, 4>(sms, g2[GEMM_V32x64])) != cudaSuccess ||
        (e = occupancy<2, 4, 2>(sms, g2[GEMM_V64x32])) != cudaSuccess ||
        (e = occupancy<2, 2, 2>(sms, g2[GEMM_V32x32])) != cudaSuccess ||
        (e = occupancy<2, 4, 4>(sms, g2[GEMM_V64x64])) != cudaSuccess)
        return e;
    return cudaSuccess;
}

cudaError_t launch_gemm1(const DQuartet* qd, const DPair* pairs, const WorkItem* items, const int* counts, double* ws,
                         int* counters, unsigned* status, cudaStream_t st) {
    (void)status;
    return launch_variants<1>(qd, pairs, items, counts, ws, ws, counters, st);
}

cudaError_t launch_gemm2(const DQuartet* qd, const DPair* pairs, const WorkItem* items, const int* counts,
                         const double* ws_in, double* out, int* counters, unsigned* status, cudaStream_t st) {
    (void)status;
    return launch_variants<2>(qd, pairs, items, counts, ws_in, out, counters, st);
}

}  // namespace lx
