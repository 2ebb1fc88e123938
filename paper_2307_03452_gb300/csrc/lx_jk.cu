// Digestion of integral blocks into Coulomb and exchange matrices (paper, Section 3: Fock
// matrix elements formed directly from the integral batches instead of storing them).  For
// quartet (ab|cd) with functions mu of a, nu of b, lam of c, sig of d:
//   J[mu][nu]  += sum_{lam, sig} (mu nu|lam sig) D[lam][sig]
//   K[mu][lam] += sum_{nu, sig}  (mu nu|lam sig) D[nu][sig]
// The blocks sit in the workspace (written there by the second transform); the kernel
// streams each once.  Every element takes part in two products, (I D_cd) for J and (I D_bd)
// for K, and on this GPU the FP64 pipe (about 1.6 FMAs per SM per clock) is the tighter
// bound, so the kernel spends as few FP64 instructions as possible beyond those two: one CTA
// per quartet, D_cd and D_bd staged in shared memory, and for each mu the threads take the
// (nu, lam) pairs, each reading its contiguous run of sig:
//   j(nu, lam) = sum_sig I[mu nu lam sig] D_cd[lam][sig]
//   k(nu, lam) = sum_sig I[mu nu lam sig] D_bd[nu][sig]
// then J[mu][nu] = sum_lam j(nu, lam) and K[mu][lam] = sum_nu k(nu, lam) are summed from
// shared memory (plain loads and adds: one add per pair and output) and added to the
// outputs with one atomic per entry.
#include <numeric>

#include "lx_internal.cuh"

namespace lx {

namespace {

constexpr int JK_THREADS = 256;
constexpr int JK_PAIRS = NCART_MAX * NCART_MAX;  // (nu, lam) pairs of one mu, at most

__global__ void __launch_bounds__(JK_THREADS) jk_digest_kernel(const DQuartet* __restrict__ qd,
                                                               const DPair* __restrict__ pairs,
                                                               const DShell* __restrict__ sh, int nquartet,
                                                               int stride,
                                                               const double* __restrict__ ws, int solid,
                                                               const double* __restrict__ D, int64_t nbf,
                                                               double* __restrict__ J, double* __restrict__ K) {
    __shared__ double Dcd[JK_PAIRS];  // [lam][sig]
    __shared__ double Dbd[JK_PAIRS];  // [nu][sig]
    __shared__ double sj[JK_PAIRS];   // j(nu, lam) of the current mu
    __shared__ double sk[JK_PAIRS];   // k(nu, lam)
    // neighbouring quartets often share a pair, and so the J or K entries they add to: CTAs
    // that run at the same time take quartets a large stride apart
    const DQuartet q = qd[(int)(((int64_t)blockIdx.x * stride) % nquartet)];
    const DPair pb = pairs[q.pb], pk = pairs[q.pk];
    const DShell sa = sh[pb.sa], sb = sh[pb.sb], sc = sh[pk.sa], sd = sh[pk.sb];
    const int na = solid ? 2 * sa.l + 1 : ncart(sa.l);
    const int nb = solid ? 2 * sb.l + 1 : ncart(sb.l);
    const int nc = solid ? 2 * sc.l + 1 : ncart(sc.l);
    const int nd = solid ? 2 * sd.l + 1 : ncart(sd.l);
    const int npair = nb * nc, tid = threadIdx.x;
    for (int i = tid; i < nc * nd; i += JK_THREADS) {
        const int l = i / nd, s = i - l * nd;
        Dcd[i] = D[(int64_t)(sc.bf + l) * nbf + sd.bf + s];
    }
    for (int i = tid; i < nb * nd; i += JK_THREADS) {
        const int n = i / nd, s = i - n * nd;
        Dbd[i] = D[(int64_t)(sb.bf + n) * nbf + sd.bf + s];
    }
    __syncthreads();
    for (int mu = 0; mu < na; ++mu) {
        const double* I = ws + q.out_off + (int64_t)mu * npair * nd;  // [nu][lam][sig]
        for (int p = tid; p < npair; p += JK_THREADS) {
            const int n = p / nc, l = p - n * nc;
            const double* run = I + (int64_t)p * nd;
            const double* dl = Dcd + l * nd;
            const double* dn = Dbd + n * nd;
            double j = 0.0, k = 0.0;
#pragma unroll 4
            for (int s = 0; s < nd; ++s) {
                const double v = __ldg(run + s);
                j = fma(v, dl[s], j);
                k = fma(v, dn[s], k);
            }
            sj[p] = j;
            sk[p] = k;
        }
        __syncthreads();
        const int64_t row = (int64_t)(sa.bf + mu) * nbf;
        if (J)
            for (int n = tid; n < nb; n += JK_THREADS) {
                double t = 0.0;
                for (int l = 0; l < nc; ++l) t += sj[n * nc + l];
                atomicAdd(&J[row + sb.bf + n], t);
            }
        if (K)
            for (int l = tid; l < nc; l += JK_THREADS) {
                double t = 0.0;
                for (int n = 0; n < nb; ++n) t += sk[n * nc + l];
                atomicAdd(&K[row + sc.bf + l], t);
            }
        __syncthreads();
    }
}

// ------------------------------------------------------------------ straight from [ab|q]
//
// With (ab|cd) = sum_k X[ab][k] H_cd[cd][k] (Eq. make-abcd), the contractions with D can be
// taken before the second transform:
//   J[mu][nu]  += sum_k X[mu nu][k] w[k],            w[k] = sum_{lam sig} H_cd[lam sig][k] D[lam][sig]
//   K[mu][lam] += sum_{nu,k} X[mu nu][k] G[nu][lam][k],  G[nu][lam][k] = sum_sig D[nu][sig] H_cd[lam sig][k]
// which costs (2 n_ab + 2 n_b n_c n_d + 2 n_a n_b n_c) K_ket N_q FLOPs per quartet instead of
// the 2 n_ab n_cd K_ket N_q of the second transform (4.3e6 against 2.6e7 for (ii|ii) solid),
// and no block is ever stored.  One CTA per quartet walks the k columns in chunks of qc:
// the chunk of X and of H_cd is staged in shared memory (rows padded to qc + 1 doubles, so
// that threads reading different rows of one column fall in different banks), w and G of
// the chunk are formed there, and each thread accumulates the J entries (mu nu) and K
// entries (mu lam) it owns in registers; one atomic per entry at the end.
constexpr int JKD_THREADS = 256;
constexpr int JKD_OWN = (NCART_MAX * NCART_MAX + JKD_THREADS - 1) / JKD_THREADS;  // entries per thread, at most

__global__ void __launch_bounds__(JKD_THREADS) jk_direct_kernel(const DQuartet* __restrict__ qd,
                                                                const DPair* __restrict__ pairs,
                                                                const DShell* __restrict__ sh, int nquartet,
                                                                int stride, int qc, const double* __restrict__ ws,
                                                                int solid, const double* __restrict__ D, int64_t nbf,
                                                                double* __restrict__ J, double* __restrict__ K) {
    extern __shared__ double jkd_smem[];
    const DQuartet q = qd[(int)(((int64_t)blockIdx.x * stride) % nquartet)];
    const DPair pb = pairs[q.pb], pk = pairs[q.pk];
    const DShell sa = sh[pb.sa], sb = sh[pb.sb], sc = sh[pk.sa], sd = sh[pk.sb];
    const int na = solid ? 2 * sa.l + 1 : ncart(sa.l);
    const int nb = solid ? 2 * sb.l + 1 : ncart(sb.l);
    const int nc = solid ? 2 * sc.l + 1 : ncart(sc.l);
    const int nd = solid ? 2 * sd.l + 1 : ncart(sd.l);
    const int nab = na * nb, ncd = nc * nd, nbc = nb * nc, nac = na * nc;
    const int K2 = q.kket * q.nq, ld = qc + 1, tid = threadIdx.x;
    double* Dcd = jkd_smem;          // [lam][sig]
    double* Dbd = Dcd + ncd;         // [nu][sig]
    double* Xs = Dbd + nb * nd;      // [nab][ld]
    double* Hs = Xs + nab * ld;      // [ncd][ld]
    double* Gs = Hs + ncd * ld;      // [nu lam][ld]
    double* wv = Gs + nbc * ld;      // [qc]
    for (int i = tid; i < ncd; i += JKD_THREADS) {
        const int l = i / nd, s = i - l * nd;
        Dcd[i] = D[(int64_t)(sc.bf + l) * nbf + sd.bf + s];
    }
    for (int i = tid; i < nb * nd; i += JKD_THREADS) {
        const int n = i / nd, s = i - n * nd;
        Dbd[i] = D[(int64_t)(sb.bf + n) * nbf + sd.bf + s];
    }
    const double* X = ws + q.x_off;    // [nab][K2]
    const double* Hc = ws + pk.h_off;  // [ncd][K2]
    double jacc[JKD_OWN], kacc[JKD_OWN];
#pragma unroll
    for (int i = 0; i < JKD_OWN; ++i) jacc[i] = kacc[i] = 0.0;
    for (int k0 = 0; k0 < K2; k0 += qc) {
        const int kc = min(qc, K2 - k0);
        __syncthreads();  // the previous chunk has been used (and D staged)
        for (int e = tid; e < nab * qc; e += JKD_THREADS) {
            const int r = e / qc, c = e - r * qc;
            Xs[r * ld + c] = c < kc ? X[(int64_t)r * K2 + k0 + c] : 0.0;
        }
        for (int e = tid; e < ncd * qc; e += JKD_THREADS) {
            const int r = e / qc, c = e - r * qc;
            Hs[r * ld + c] = c < kc ? Hc[(int64_t)r * K2 + k0 + c] : 0.0;
        }
        __syncthreads();
        if (J)
            for (int c = tid; c < qc; c += JKD_THREADS) {
                double w = 0.0;
                for (int i = 0; i < ncd; ++i) w = fma(Hs[i * ld + c], Dcd[i], w);
                wv[c] = w;
            }
        if (K)  // G only for K (J alone costs 4 n_ab K_ket N_q FLOPs per quartet)
            for (int e = tid; e < nbc * qc; e += JKD_THREADS) {
                const int nl = e / qc, c = e - nl * qc, n = nl / nc, l = nl - n * nc;
                const double* dn = Dbd + n * nd;
                const double* hl = Hs + (l * nd) * ld + c;
                double g = 0.0;
                for (int s = 0; s < nd; ++s) g = fma(dn[s], hl[s * ld], g);
                Gs[nl * ld + c] = g;
            }
        __syncthreads();
#pragma unroll
        for (int i = 0; i < JKD_OWN; ++i) {
            const int r = tid + i * JKD_THREADS;
            if (J && r < nab) {
                const double* xr = Xs + r * ld;
                double t = jacc[i];
                for (int c = 0; c < qc; ++c) t = fma(xr[c], wv[c], t);
                jacc[i] = t;
            }
            const int o = tid + i * JKD_THREADS;
            if (K && o < nac) {
                const int m = o / nc, l = o - m * nc;
                double t = kacc[i];
                for (int n = 0; n < nb; ++n) {
                    const double* xr = Xs + (m * nb + n) * ld;
                    const double* gr = Gs + (n * nc + l) * ld;
                    for (int c = 0; c < qc; ++c) t = fma(xr[c], gr[c], t);
                }
                kacc[i] = t;
            }
        }
    }
#pragma unroll
    for (int i = 0; i < JKD_OWN; ++i) {
        const int r = tid + i * JKD_THREADS;
        if (J && r < nab) {
            const int m = r / nb, n = r - m * nb;
            atomicAdd(&J[(int64_t)(sa.bf + m) * nbf + sb.bf + n], jacc[i]);
        }
        if (K && r < nac) {
            const int m = r / nc, l = r - m * nc;
            atomicAdd(&K[(int64_t)(sa.bf + m) * nbf + sc.bf + l], kacc[i]);
        }
    }
}

}  // namespace

// shared memory of jk_direct_kernel for the given sizes and chunk width qc
size_t jk_direct_smem(int nab, int ncd, int nb, int nc, int nd, int qc) {
    return sizeof(double) * ((size_t)ncd + (size_t)nb * nd + (size_t)(nab + ncd + nb * nc) * (qc + 1) + qc);
}

cudaError_t launch_jk_direct(const DQuartet* qd, const DPair* pairs, const DShell* sh, int nquartet, int qc,
                             size_t smem, const double* ws, bool solid, const double* D, int64_t nbf, double* J,
                             double* K, cudaStream_t st) {
    if (nquartet <= 0 || (!J && !K)) return cudaSuccess;
    if (qc < 1 || smem > JKD_SMEM_MAX) return cudaErrorInvalidValue;
    int stride = 7919;  // prime; coprime with nquartet, so the map below is a permutation
    while (nquartet > 1 && std::gcd(stride, nquartet) != 1) stride += 2;
    jk_direct_kernel<<<nquartet, JKD_THREADS, smem, st>>>(qd, pairs, sh, nquartet, stride, qc, ws, solid ? 1 : 0, D,
                                                          nbf, J, K);
    return cudaGetLastError();
}

cudaError_t init_jk_kernels() {
    return cudaFuncSetAttribute(jk_direct_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)JKD_SMEM_MAX);
}

cudaError_t launch_jk_digest(const DQuartet* qd, const DPair* pairs, const DShell* sh, int nquartet,
                             const double* ws, bool solid, const double* D, int64_t nbf, double* J, double* K,
                             cudaStream_t st) {
    if (nquartet <= 0 || (!J && !K)) return cudaSuccess;
    int stride = 7919;  // prime; coprime with nquartet, so the map below is a permutation
    while (nquartet > 1 && std::gcd(stride, nquartet) != 1) stride += 2;
    jk_digest_kernel<<<nquartet, JK_THREADS, 0, st>>>(qd, pairs, sh, nquartet, stride, ws, solid ? 1 : 0, D, nbf, J,
                                                      K);
    return cudaGetLastError();
}

}  // namespace lx
