// Shell-pair preparation: contraction normalisation and the Hermite-to-Cartesian/solid
// matrices H of each primitive pair (paper, Section 2: the Gaussian product after
// Eq. cart2herm-2, the E recursions, and the definition of H).
#include <cmath>

#include "lx_internal.cuh"

namespace lx {

namespace {

constexpr int NSOLID_PACKED = 840;  // sum over l = 0..6 of (2l+1) ncart(l)
__constant__ double c_solid[NSOLID_PACKED];
__constant__ int c_solid_off[LMAX + 2];
__device__ int g_tuv_prep[NHERM_TOT];
__constant__ SolidClassTab c_cls[LMAX + 1];

constexpr double PI = 3.141592653589793238462643383279502884;

__device__ inline void set_status(unsigned* st, unsigned bit) { atomicOr(st, bit); }

// Cartesian exponents of component k of shell l: i = l - ax runs 0..l, j = az runs 0..i.
__device__ inline void cart_of(int k, int l, int& ax, int& ay, int& az) {
    int i = (int)((sqrtf(8.0f * k + 1.0f) - 1.0f) * 0.5f);
    while ((i + 1) * (i + 2) / 2 <= k) ++i;
    while (i * (i + 1) / 2 > k) --i;
    az = k - i * (i + 1) / 2;
    ay = i - az;
    ax = l - i;
}

// (2n-1)!!
__device__ inline double dfact_odd(int n) {
    double r = 1.0;
    for (int k = 2 * n - 1; k > 1; k -= 2) r *= k;
    return r;
}

// Normaliser of x^l exp(-zeta r^2): (2 zeta/pi)^{3/4} (4 zeta)^{l/2} / sqrt((2l-1)!!).
__device__ inline double prim_norm(int l, double z) {
    return pow(2.0 * z / PI, 0.75) * pow(4.0 * z, 0.5 * l) / sqrt(dfact_odd(l));
}

// One thread per shell: c'_i = c_i N(zeta_i, l) s, with s making the contracted x^l
// function unit-normalised: sum_ij c'_i c'_j (2l-1)!! / (2(z_i+z_j))^l (pi/(z_i+z_j))^{3/2} = 1.
__global__ void norm_kernel(const DShell* __restrict__ sh, int nshell, const double* __restrict__ exps,
                            const double* __restrict__ coefs, double* __restrict__ ncoef, unsigned* status) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nshell) return;
    const DShell d = sh[s];
    const int l = d.l, K = d.K, o = d.prim_off;
    double acc = 0.0;
    const double df = dfact_odd(l);
    for (int i = 0; i < K; ++i)
        for (int j = 0; j < K; ++j) {
            const double zi = exps[o + i], zj = exps[o + j], ab = zi + zj;
            const double ov = df / pow(2.0 * ab, l) * pow(PI / ab, 1.5);
            acc += coefs[o + i] * coefs[o + j] * prim_norm(l, zi) * prim_norm(l, zj) * ov;
        }
    if (!(acc > 0.0)) set_status(status, ST_BAD_INPUT);
    const double sc = 1.0 / sqrt(acc);
    for (int i = 0; i < K; ++i) ncoef[o + i] = coefs[o + i] * prim_norm(l, exps[o + i]) * sc;
}

// Solid fold of one (class of a, class of b, p) item with exactly NMA x NMB solid functions:
// for each a of the class, u[jb] = sum_b C_b[jb][b] E_ab^p over the class of b (the E product
// formed once per b), then acc[ja][jb] += C_a[ja][a] u[jb].  The class sizes are template
// arguments so that no padded FP64 operation is issued.
template <int NMA, int NMB>
__device__ inline void fold_item(const SolidClassTab& TA, const SolidClassTab& TB, int ca, int cb, int px, int py,
                                 int pz, const double* Ex, const double* Ey, const double* Ez, int sb1, int nt,
                                 double (&out)[SC_MAXM][SC_MAXM]) {
    double acc[NMA][NMB];
#pragma unroll
    for (int x = 0; x < NMA; ++x)
#pragma unroll
        for (int y = 0; y < NMB; ++y) acc[x][y] = 0.0;
    const int na = TA.na[ca], nb = TB.na[cb];
    for (int ia = 0; ia < na; ++ia) {
        const int ac = TA.comp[ca][ia];
        const double* ex = Ex + ((ac & 255) * sb1) * nt + px;
        const double* ey = Ey + (((ac >> 8) & 255) * sb1) * nt + py;
        const double* ez = Ez + ((ac >> 16) * sb1) * nt + pz;
        double u[NMB];
#pragma unroll
        for (int y = 0; y < NMB; ++y) u[y] = 0.0;
        for (int ib = 0; ib < nb; ++ib) {
            const int bc = TB.comp[cb][ib];
            const double v = ex[(bc & 255) * nt] * ey[((bc >> 8) & 255) * nt] * ez[(bc >> 16) * nt];
#pragma unroll
            for (int y = 0; y < NMB; ++y) u[y] += TB.c[cb][y][ib] * v;
        }
#pragma unroll
        for (int x = 0; x < NMA; ++x) {
            const double c = TA.c[ca][x][ia];
#pragma unroll
            for (int y = 0; y < NMB; ++y) acc[x][y] += c * u[y];
        }
    }
#pragma unroll
    for (int x = 0; x < NMA; ++x)
#pragma unroll
        for (int y = 0; y < NMB; ++y) out[x][y] = acc[x][y];
}

constexpr int PAIR_THREADS = 128;
constexpr int ETAB = (LMAX + 1) * (LMAX + 1) * (2 * LMAX + 1);  // 637 per direction

// One CTA per primitive pair (item.q = pair id, item.a = primitive pair kp).
// Writes pair scalars (zeta_p, P) and the H block columns of this primitive pair.
__global__ void __launch_bounds__(PAIR_THREADS) pair_h_kernel(const DPair* __restrict__ pairs,
                                                               const WorkItem* __restrict__ items,
                                                               const DShell* __restrict__ sh,
                                                               const double* __restrict__ exps,
                                                               const double* __restrict__ ncoef,
                                                               double* __restrict__ ws, double* __restrict__ ws_info,
                                                               unsigned* status) {
    __shared__ double E[3][ETAB];
    __shared__ double s_pref;
    const WorkItem it = items[blockIdx.x];
    const DPair pr = pairs[it.q];
    const DShell sa = sh[pr.sa], sb = sh[pr.sb];
    const int la = sa.l, lb = sb.l, lsum = la + lb, nt = lsum + 1;
    const int kp = it.a, ia = kp / sb.K, ib = kp - ia * sb.K;
    const double za = exps[sa.prim_off + ia], zb = exps[sb.prim_off + ib], zp = za + zb;

    for (int i = threadIdx.x; i < 3 * ETAB; i += blockDim.x) (&E[0][0])[i] = 0.0;
    __syncthreads();
    // Hermite expansion coefficients, one warp per Cartesian direction, lanes over t:
    //   E^t_{i+1,j} = E^{t-1}_{ij}/(2 zeta_p) + (P - A) E^t_{ij} + (t+1) E^{t+1}_{ij}
    //   E^t_{i,j+1} = E^{t-1}_{ij}/(2 zeta_p) + (P - B) E^t_{ij} + (t+1) E^{t+1}_{ij}
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (warp < 3) {
        const int d = warp;
        const double Ad = sh[pr.sa].A[d], Bd = sh[pr.sb].A[d];
        const double P = (za * Ad + zb * Bd) / zp;
        const double PA = P - Ad, PB = P - Bd, oo2p = 0.5 / zp;
        double* Ed = E[d];
#define EIJ(i, j, t) Ed[((i) * (lb + 1) + (j)) * nt + (t)]
        if (lane == 0) EIJ(0, 0, 0) = 1.0;
        __syncwarp();
        for (int i = 0; i <= la; ++i) {
            if (i > 0) {
                const int t = lane;
                double v = 0.0;
                if (t <= i) {
                    v = PA * EIJ(i - 1, 0, t);
                    if (t > 0) v += oo2p * EIJ(i - 1, 0, t - 1);
                    if (t + 1 <= i - 1) v += (t + 1) * EIJ(i - 1, 0, t + 1);
                }
                __syncwarp();
                if (t <= i) EIJ(i, 0, t) = v;
                __syncwarp();
            }
            for (int j = 1; j <= lb; ++j) {
                const int t = lane;
                double v = 0.0;
                if (t <= i + j) {
                    if (t <= i + j - 1) v = PB * EIJ(i, j - 1, t);
                    if (t > 0) v += oo2p * EIJ(i, j - 1, t - 1);
                    if (t + 1 <= i + j - 1) v += (t + 1) * EIJ(i, j - 1, t + 1);
                }
                __syncwarp();
                if (t <= i + j) EIJ(i, j, t) = v;
                __syncwarp();
            }
        }
#undef EIJ
    } else if (threadIdx.x == 96) {
        // pair scalars and the prefactor exp(-mu |AB|^2) c'_a c'_b
        double AB2 = 0.0;
        double* info = ws_info + pr.info_off + 4 * (int64_t)kp;
        info[0] = zp;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            info[1 + d] = (za * sa.A[d] + zb * sb.A[d]) / zp;
            AB2 += (sa.A[d] - sb.A[d]) * (sa.A[d] - sb.A[d]);
        }
        s_pref = exp(-za * zb / zp * AB2) * ncoef[sa.prim_off + ia] * ncoef[sb.prim_off + ib];
    }
    __syncthreads();

    const int np = pr.np;
    const int64_t ldh = (int64_t)pr.Kab * np;
    double* H = ws + pr.h_off + (int64_t)kp * np;
    const double pref = s_pref;
    const int nca = ncart(la), ncb = ncart(lb);
    const double* Ex = E[0];
    const double* Ey = E[1];
    const double* Ez = E[2];
    const int sb1 = lb + 1;

    if (!pr.solid) {
        // H[ab][p] = pref * sign(p) * Ex[ax bx px] Ey[ay by py] Ez[az bz pz]
        const int total = nca * ncb * np;
        for (int i = threadIdx.x; i < total; i += blockDim.x) {
            const int ab = i / np, p = i - ab * np;
            const int a = ab / ncb, b = ab - a * ncb;
            int ax, ay, az, bx, by, bz;
            cart_of(a, la, ax, ay, az);
            cart_of(b, lb, bx, by, bz);
            const int tuv = g_tuv_prep[p];
            const int px = tuv & 255, py = (tuv >> 8) & 255, pz = tuv >> 16;
            double v = Ex[(ax * sb1 + bx) * nt + px] * Ey[(ay * sb1 + by) * nt + py] * Ez[(az * sb1 + bz) * nt + pz];
            if (pr.sign && ((px + py + pz) & 1)) v = -v;
            H[(int64_t)ab * ldh + p] = pref * v;
        }
    } else {
        // H[ma mb][p] = pref * sign(p) * sum_a C_a[ma][a] sum_b C_b[mb][b] E_ab^p.
        // C is block diagonal over parity classes, so one work item is (class of a, class of
        // b, p): the E products of the class's b components are formed once per a and shared
        // by all of its m_b; the a-sum accumulates a (<= 4) x (<= 4) register block.
        const SolidClassTab& TA = c_cls[la];
        const SolidClassTab& TB = c_cls[lb];
        const int nsb = 2 * lb + 1;
        const int ncb_cls = TB.ncls;
        const int total = TA.ncls * ncb_cls * np;
        for (int i = threadIdx.x; i < total; i += blockDim.x) {
            const int g = i / np, p = i - g * np;
            const int ca = g / ncb_cls, cb = g - ca * ncb_cls;
            const int tuv = g_tuv_prep[p];
            const int px = tuv & 255, py = (tuv >> 8) & 255, pz = tuv >> 16;
            const int nma = TA.nm[ca], nmb = TB.nm[cb];
            double acc[SC_MAXM][SC_MAXM];
#define LX_FOLD(A, B) \
    case (A) * 8 + (B): fold_item<A, B>(TA, TB, ca, cb, px, py, pz, Ex, Ey, Ez, sb1, nt, acc); break;
            switch (nma * 8 + nmb) {
                LX_FOLD(1, 1) LX_FOLD(1, 2) LX_FOLD(1, 3) LX_FOLD(1, 4)
                LX_FOLD(2, 1) LX_FOLD(2, 2) LX_FOLD(2, 3) LX_FOLD(2, 4)
                LX_FOLD(3, 1) LX_FOLD(3, 2) LX_FOLD(3, 3) LX_FOLD(3, 4)
                LX_FOLD(4, 1) LX_FOLD(4, 2) LX_FOLD(4, 3) LX_FOLD(4, 4)
                default: break;
            }
#undef LX_FOLD
            const double sg = (pr.sign && ((px + py + pz) & 1)) ? -pref : pref;
#pragma unroll
            for (int ja = 0; ja < SC_MAXM; ++ja)
#pragma unroll
                for (int jb = 0; jb < SC_MAXM; ++jb)
                    if (ja < nma && jb < nmb)
                        H[(int64_t)(TA.mind[ca][ja] * nsb + TB.mind[cb][jb]) * ldh + p] = sg * acc[ja][jb];
        }
    }
}

}  // namespace

cudaError_t init_prep_tables(const double* host_coefs, const int* host_tuv, const void* host_classes) {
    int off[LMAX + 2];
    off[0] = 0;
    for (int l = 0; l <= LMAX; ++l) off[l + 1] = off[l] + (2 * l + 1) * ncart(l);
    if (off[LMAX + 1] != NSOLID_PACKED) return cudaErrorInvalidValue;
    cudaError_t e = cudaMemcpyToSymbol(c_solid, host_coefs, sizeof(double) * NSOLID_PACKED);
    if (e != cudaSuccess) return e;
    e = cudaMemcpyToSymbol(c_solid_off, off, sizeof(off));
    if (e != cudaSuccess) return e;
    e = cudaMemcpyToSymbol(c_cls, host_classes, sizeof(SolidClassTab) * (LMAX + 1));
    if (e != cudaSuccess) return e;
    return cudaMemcpyToSymbol(g_tuv_prep, host_tuv, sizeof(int) * NHERM_TOT);
}

cudaError_t launch_norm(const DShell* sh, int nshell, const double* exps, const double* coefs, double* ncoef,
                        unsigned* status, cudaStream_t st) {
    if (nshell <= 0) return cudaSuccess;
    norm_kernel<<<(nshell + 127) / 128, 128, 0, st>>>(sh, nshell, exps, coefs, ncoef, status);
    return cudaGetLastError();
}

cudaError_t launch_pair_h(const DPair* pairs, const WorkItem* items, int nitems, const DShell* sh,
                          const double* exps, const double* ncoef, double* ws, double* ws_info, unsigned* status,
                          cudaStream_t st) {
    if (nitems <= 0) return cudaSuccess;
    pair_h_kernel<<<nitems, PAIR_THREADS, 0, st>>>(pairs, items, sh, exps, ncoef, ws, ws_info, status);
    return cudaGetLastError();
}

}  // namespace lx
