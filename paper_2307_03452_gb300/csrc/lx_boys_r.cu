// Boys function (Eq. boys) and the auxiliary Hermite integrals [r]^(m) (Eq. md1).
//
// Boys: for T < 36, F_mmax(T) from an 8-term Taylor expansion around the nearest point
// of a 0.1-spaced table of F_n(T_k), then the downward recursion
// F_m = (2T F_{m+1} + exp(-T)) / (2m+1); for T >= 36, F_0 = (1/2) sqrt(pi/T) (erf(sqrt T)
// differs from 1 by < 3e-17) and the upward recursion F_{m+1} = ((2m+1) F_m - exp(-T))/(2T).
//
// R: one warp per primitive quartet evaluates [r]^(m) for m = L-1 down to 0 in one shared
// array of pyr(L) doubles, overwriting [r]^(m+1) with [r]^(m) (the paper's in-place
// scheme, Section 3): within level m the totals n = |r| are processed from L-m down
// to 1, so the inputs at totals n-1 and n-2 still hold level m+1 when they are read.
// In the batch kernel each CTA is that one warp, with shared memory for the chunk's
// largest L, so that as many quartets as shared memory allows run side by side.
#include <cmath>
#include <cstring>
#include <vector>

#include "lx_internal.cuh"

namespace lx {

namespace {

__device__ double g_boys[BOYS_NROW * BOYS_NPT];
// One step of Eq. md1 for every Hermite position h = hidx(t, u, v) with t + u + v >= 1,
// lowering the first nonzero direction d of (t, u, v):
//   [r]^(m) = X_d [r - 1_d]^(m+1) + (r_d - 1) [r - 2_d]^(m+1)
// x = hidx(r - 1_d) | hidx(r - 2_d) << 13 | d << 26 (the second position 0 when r_d = 1),
// (z, w) = the FP64 bits of r_d - 1 (low, high word), so that the step is one multiply and one
// FMA with no branch and no integer conversion.
__device__ int4 g_rec[NHERM_TOT];

constexpr double PI = 3.141592653589793238462643383279502884;

__device__ inline void set_status(unsigned* st, unsigned bit) { atomicOr(st, bit); }

// F_m(T) for m = 0..mmax (mmax <= LTOT) into F (any memory), one thread.
__device__ void boys_eval(int mmax, double T, double* F) {
    if (T < BOYS_TMAX) {
        const int k = __double2int_rn(T * (1.0 / BOYS_DT));
        const double d = k * BOYS_DT - T;  // -(T - T_k)
        // F_mmax(T) = sum_j F_{mmax+j}(T_k) (-(T - T_k))^j / j!
        const double* col = g_boys + k;
        double f = 0.0, pw = 1.0;
#pragma unroll
        for (int j = 0; j < BOYS_ORDER; ++j) {
            f += __ldg(col + (mmax + j) * BOYS_NPT) * pw;
            pw *= d / (j + 1);
        }
        F[mmax] = f;
        const double e = exp(-T), twoT = 2.0 * T;
        for (int m = mmax - 1; m >= 0; --m) {
            f = (twoT * f + e) / (2 * m + 1);
            F[m] = f;
        }
    } else {
        double f = 0.5 * sqrt(PI / T);
        F[0] = f;
        const double e = exp(-T), oo2T = 0.5 / T;
        for (int m = 0; m < mmax; ++m) {
            f = ((2 * m + 1) * f - e) * oo2T;
            F[m + 1] = f;
        }
    }
}

// B[m] *= pref (-2 rho)^m for m = 0..L (L <= LTOT < 32), one m per lane: the power is
// taken directly rather than as a running product, which keeps its rounding at one step.
__device__ inline void scale_base(int L, double rho, double pref, double* B, int lane) {
    if (lane <= L) {
        const double pw = pow(2.0 * rho, (double)lane);
        B[lane] *= (lane & 1) ? -pref * pw : pref * pw;
    }
}

// In-place Eq. md1 on R[pyr(L)] (shared memory), by one warp.  B[m] = [0]^(m), m = 0..L.
// On return R holds [r]^(0).
__device__ void hermite_r_warp(int L, double X, double Y, double Z, const double* B, double* R, int lane) {
    if (lane == 0) R[0] = B[L];
    __syncwarp();
    for (int m = L - 1; m >= 0; --m) {
        for (int n = L - m; n >= 1; --n) {
            const int base = n * (n + 1) * (n + 2) / 6;  // pyr(n-1)
            const int cnt = (n + 1) * (n + 2) / 2;
            for (int s = lane; s < cnt; s += 32) {
                const int4 e = __ldg(&g_rec[base + s]);
                const int d = e.x >> 26;
                const double xd = d == 0 ? X : (d == 1 ? Y : Z);
                R[base + s] = fma(__hiloint2double(e.w, e.z), R[(e.x >> 13) & 0x1FFF], xd * R[e.x & 0x1FFF]);
            }
            __syncwarp();
        }
        if (lane == 0) R[0] = B[m];
        __syncwarp();
    }
}

constexpr int BR_WARPS = 4;  // warps per CTA of the stage entry point

// One single-warp CTA per primitive quartet: item.q = quartet, item.a = kpq = kp * kket + kq.
__global__ void __launch_bounds__(32) boys_r_kernel(const DQuartet* __restrict__ qd, const DPair* __restrict__ pairs,
                                                    const WorkItem* __restrict__ items, double* __restrict__ ws,
                                                    unsigned* status) {
    extern __shared__ double smem[];
    const int lane = threadIdx.x & 31;
    const WorkItem it = items[blockIdx.x];
    const DQuartet q = qd[it.q];
    const int kpq = it.a;
    const int nr = q.nr;
    double* R = smem;
    double* B = R + nr;
    const int kp = kpq / q.kket, kq = kpq - kp * q.kket;
    const DPair pb = pairs[q.pb], pk = pairs[q.pk];
    const double* ib = ws + pb.info_off + 4 * (int64_t)kp;
    const double* ik = ws + pk.info_off + 4 * (int64_t)kq;
    const double zp = ib[0], zq = ik[0];
    const double X = ib[1] - ik[1], Y = ib[2] - ik[2], Z = ib[3] - ik[3];
    const double rho = zp * zq / (zp + zq);
    const double T = rho * (X * X + Y * Y + Z * Z);
    if (lane == 0) boys_eval(q.L, T, B);
    __syncwarp();
    // [0]^(m) = (-2 rho)^m 2 pi^{5/2} / (zeta_p zeta_q sqrt(zeta_p + zeta_q)) F_m(T), one m per lane
    scale_base(q.L, rho, 2.0 * PI * PI * sqrt(PI) / (zp * zq * sqrt(zp + zq)), B, lane);
    __syncwarp();
    hermite_r_warp(q.L, X, Y, Z, B, R, lane);
    double* out = ws + q.rr_off + (int64_t)kpq * nr;
    for (int r = lane; r < nr; r += 32) out[r] = R[r];
}

__global__ void boys_stage_kernel(int mmax, const double* __restrict__ T, int64_t n, double* __restrict__ F,
                                  unsigned* status) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double t = T[i];
    double buf[LTOT + 1];
    if (!(t >= 0.0) || !isfinite(t)) {
        set_status(status, ST_BAD_INPUT);
        for (int m = 0; m <= mmax; ++m) F[i * (mmax + 1) + m] = nan("");
        return;
    }
    boys_eval(mmax, t, buf);
    for (int m = 0; m <= mmax; ++m) F[i * (mmax + 1) + m] = buf[m];
}

// Stage entry: params[5i..] = (rho, X, Y, Z, pref) -> R[i * pyr(L) ..].
__global__ void __launch_bounds__(BR_WARPS * 32) hermite_r_stage_kernel(int L, const double* __restrict__ params,
                                                                        int64_t n, double* __restrict__ Rout) {
    extern __shared__ double smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t item = (int64_t)blockIdx.x * BR_WARPS + warp;
    if (item >= n) return;
    const int nr = pyr(L);
    double* R = smem + warp * (nr + LTOT + 1);
    double* B = R + nr;
    const double rho = params[5 * item], X = params[5 * item + 1], Y = params[5 * item + 2],
                 Z = params[5 * item + 3], pref = params[5 * item + 4];
    if (lane == 0) boys_eval(L, rho * (X * X + Y * Y + Z * Z), B);
    __syncwarp();
    scale_base(L, rho, pref, B, lane);
    __syncwarp();
    hermite_r_warp(L, X, Y, Z, B, R, lane);
    for (int r = lane; r < nr; r += 32) Rout[item * nr + r] = R[r];
}

size_t br_smem(int L) { return sizeof(double) * BR_WARPS * (size_t)(pyr(L) + LTOT + 1); }

}  // namespace

cudaError_t init_boys_table(const double* host_table) {
    cudaError_t e = cudaMemcpyToSymbol(g_boys, host_table, sizeof(double) * BOYS_NROW * BOYS_NPT);
    if (e != cudaSuccess) return e;
    static_assert(NHERM_TOT <= 8192, "Hermite positions fit 13 bits");
    std::vector<int4> rec(NHERM_TOT, make_int4(0, 0, 0, 0));
    for (int n = 1; n <= LTOT; ++n)
        for (int i = 0; i <= n; ++i)
            for (int v = 0; v <= i; ++v) {
                const int u = i - v, t = n - i;
                const int d = t > 0 ? 0 : (u > 0 ? 1 : 2), rd = d == 0 ? t : (d == 1 ? u : v);
                const int dt = d == 0, du = d == 1, dv = d == 2;
                const int h1 = hidx(t - dt, u - du, v - dv);
                const int h2 = rd > 1 ? hidx(t - 2 * dt, u - 2 * du, v - 2 * dv) : 0;
                const double c = rd - 1;
                long long bits;
                std::memcpy(&bits, &c, sizeof(bits));
                rec[hidx(t, u, v)] = make_int4(h1 | (h2 << 13) | (d << 26), 0, (int)(bits & 0xFFFFFFFFll), (int)(bits >> 32));
            }
    if ((e = cudaMemcpyToSymbol(g_rec, rec.data(), sizeof(int4) * NHERM_TOT)) != cudaSuccess) return e;
    e = cudaFuncSetAttribute(boys_r_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(sizeof(double) * (pyr(LTOT) + LTOT + 1)));
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(hermite_r_stage_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)br_smem(LTOT));
}

cudaError_t launch_boys_r(const DQuartet* qd, const DPair* pairs, const WorkItem* items, int nitems, int lmax,
                          double* ws, unsigned* status, cudaStream_t st) {
    if (nitems <= 0) return cudaSuccess;
    if (lmax < 0 || lmax > LTOT) return cudaErrorInvalidValue;
    const size_t smem = sizeof(double) * (pyr(lmax) + LTOT + 1);
    boys_r_kernel<<<nitems, 32, smem, st>>>(qd, pairs, items, ws, status);
    return cudaGetLastError();
}

cudaError_t launch_boys(int mmax, const double* T, int64_t n, double* F, unsigned* status, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    boys_stage_kernel<<<(unsigned)((n + 127) / 128), 128, 0, st>>>(mmax, T, n, F, status);
    return cudaGetLastError();
}

cudaError_t launch_hermite_r(int L, const double* params, int64_t n, double* R, unsigned* status, cudaStream_t st) {
    (void)status;
    if (n <= 0) return cudaSuccess;
    hermite_r_stage_kernel<<<(unsigned)((n + BR_WARPS - 1) / BR_WARPS), BR_WARPS * 32, br_smem(L), st>>>(L, params,
                                                                                                          n, R);
    return cudaGetLastError();
}

}  // namespace lx
