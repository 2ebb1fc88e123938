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

}  // namespace

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
