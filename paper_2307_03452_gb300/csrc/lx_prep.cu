// Shell-pair preparation: contraction normalisation and the Hermite-to-Cartesian/solid
// matrices H of each primitive pair (paper, Section 2: the Gaussian product after
// Eq. cart2herm-2, the E recursions, and the definition of H).
#include <algorithm>
#include <cmath>

#include "lx_internal.cuh"

namespace lx {

namespace {

__constant__ double c_solid[NSOLID_PACKED];
__constant__ int c_solid_off[LMAX + 2];
__device__ int g_tuv_prep[NHERM_TOT];

struct FoldDev {
    const int *q_ent, *w_ent, *h_ent, *h_out, *wstart, *g_rec;
    const FoldSeg* segs;
    FoldPairTab pair[LMAX + 1][LMAX + 1];
};
__constant__ FoldDev c_fold;

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

constexpr int PAIR_THREADS = 128;
constexpr int PAIR_SOLID_THREADS = 32 * FOLD_NWARP;  // one fold stream per warp
// E entries per Cartesian direction of a pair with la, lb <= l: (l+1)^2 (2l+1)
__host__ __device__ constexpr int etab_of(int l) { return (l + 1) * (l + 1) * (2 * l + 1); }
// solid-harmonic coefficients of one shell of angular momentum l: (2l+1) ncart(l)
__host__ __device__ constexpr int ncoef_of(int l) { return (2 * l + 1) * (l + 1) * (l + 2) / 2; }
constexpr int ETAB = etab_of(LMAX);  // 960 per direction
// shared memory of pair_h_solid_kernel for pairs with la, lb <= lcap and fold capacities qcap
// (Q rows incl. the zero row), wcap and gcap (G entries incl. the zero): E[3][etab], C_a and
// C_b (each with a trailing zero), Q, W, G, then one int per Hermite index of the pair (column
// exponents)
inline size_t fold_smem_bytes(int lcap, int qcap, int wcap, int gcap) {
    return sizeof(double) * (size_t)(3 * etab_of(lcap) + 2 * (ncoef_of(lcap) + 1) + qcap + wcap + gcap) +
           sizeof(int) * (size_t)pyr(2 * lcap);
}

// Hermite expansion coefficients of primitive pair kp into E[3][etab] (zero beyond t <= i+j),
// one warp per Cartesian direction, lanes over t:
//   E^t_{i+1,j} = E^{t-1}_{ij}/(2 zeta_p) + (P - A) E^t_{ij} + (t+1) E^{t+1}_{ij}
//   E^t_{i,j+1} = E^{t-1}_{ij}/(2 zeta_p) + (P - B) E^t_{ij} + (t+1) E^{t+1}_{ij}
// Thread 96 writes the pair scalars (zeta_p, P) and leaves exp(-mu |AB|^2) c'_a c'_b in
// *s_pref.  Needs at least 97 threads; ends with a CTA barrier.
__device__ __forceinline__ void pair_setup(const DPair& pr, int kp, const DShell* __restrict__ sh, const double* __restrict__ exps,
                           const double* __restrict__ ncoef, double* __restrict__ ws_info, double* E,
                           int etab, double* s_pref) {
    const DShell sa = sh[pr.sa], sb = sh[pr.sb];
    const int la = sa.l, lb = sb.l, nt = la + lb + 1;
    const int ia = kp / sb.K, ib = kp - ia * sb.K;
    const double za = exps[sa.prim_off + ia], zb = exps[sb.prim_off + ib], zp = za + zb;
    for (int i = threadIdx.x; i < 3 * etab; i += blockDim.x) E[i] = 0.0;
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (warp < 3) {
        const int d = warp;
        const double Ad = sh[pr.sa].A[d], Bd = sh[pr.sb].A[d];
        const double P = (za * Ad + zb * Bd) / zp;
        const double PA = P - Ad, PB = P - Bd, oo2p = 0.5 / zp;
        double* Ed = E + d * etab;
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
        *s_pref = exp(-za * zb / zp * AB2) * ncoef[sa.prim_off + ia] * ncoef[sb.prim_off + ib];
    }
    __syncthreads();
}

// Largest exponent field of the values stored in each column (shared-memory maxima), turned
// into the column scales c_k (|x| < 2^c_k over the column, 0 for a zero column) of the split
// path.
__device__ inline int exp_field_of(double v) { return (int)((__double_as_longlong(v) >> 52) & 0x7FF); }
__device__ inline void write_col_scales(const int* cexp, int np, int* out) {
    for (int p = threadIdx.x; p < np; p += blockDim.x) out[p] = cexp[p] > 0 ? cexp[p] - 1022 : 0;
}

// One CTA per primitive pair (item.q = pair id, item.a = primitive pair kp), Cartesian rows.
// Writes pair scalars (zeta_p, P) and the H block columns of this primitive pair (and, on the
// split path, their column scales).
__global__ void __launch_bounds__(PAIR_THREADS) pair_h_kernel(const DPair* __restrict__ pairs,
                                                               const WorkItem* __restrict__ items,
                                                               const DShell* __restrict__ sh,
                                                               const double* __restrict__ exps,
                                                               const double* __restrict__ ncoef,
                                                               double* __restrict__ ws, double* __restrict__ ws_info,
                                                               unsigned* status) {
    __shared__ double E[3][ETAB];
    __shared__ double s_pref;
    __shared__ int cexp[NHERM_PAIR];
    const WorkItem it = items[blockIdx.x];
    const DPair pr = pairs[it.q];
    const int la = sh[pr.sa].l, lb = sh[pr.sb].l, nt = la + lb + 1;
    const int kp = it.a;
    const bool scales = pr.cs_off >= 0;
    for (int p = threadIdx.x; p < pr.np; p += blockDim.x) cexp[p] = 0;  // ordered by pair_setup's barriers
    pair_setup(pr, kp, sh, exps, ncoef, ws_info, &E[0][0], ETAB, &s_pref);

    const int np = pr.np;
    const int64_t ldh = (int64_t)pr.Kab * np;
    double* H = ws + pr.h_off + (int64_t)kp * np;
    const double pref = s_pref;
    const int nca = ncart(la), ncb = ncart(lb);
    const double* Ex = E[0];
    const double* Ey = E[1];
    const double* Ez = E[2];
    const int sb1 = lb + 1;

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
        const double h = pref * v;
        H[(int64_t)ab * ldh + p] = h;
        if (scales) atomicMax(&cexp[p], exp_field_of(h));
    }
    if (scales) {
        __syncthreads();
        write_col_scales(cexp, np, reinterpret_cast<int*>(reinterpret_cast<char*>(ws) + pr.cs_off) + (int64_t)kp * np);
    }
}

// One fold stage (row layout with FoldSeg).  Each warp walks its own stream of entry quads,
// three 16-byte loads ahead, summing term(entry) into the row it holds (lane i: row 32 g + i,
// g = fold_group(k, warp) in round k).  A flagged column ends the group: the warp stores its
// rows with the value pre(row) fetched one group earlier (rows >= nrow store nothing) and
// goes on to round k + 1.  Rows are short (1.4 to 2.3 entries on average for l = 6 pairs), so
// no load of the stream waits on another.
template <typename Term, typename Pre, typename Store>
__device__ __forceinline__ void fold_stage(int ws, int nrow, const int* __restrict__ ent, Term term, Pre pre,
                                           Store store) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int s0 = __ldg(&c_fold.wstart[ws + warp]), s1 = __ldg(&c_fold.wstart[ws + warp + 1]);
    const int4* src = reinterpret_cast<const int4*>(ent + s0) + lane;
    const int nq = (s1 - s0) >> 7;
    int k = 0, r = 32 * fold_group(0, warp) + lane;
    int ck = pre(r), nk = pre(32 * fold_group(1, warp) + lane);
    const int4 z = make_int4(0, 0, 0, 0);
    int4 e0 = nq > 0 ? __ldg(src) : z, e1 = nq > 1 ? __ldg(src + 32) : z, e2 = nq > 2 ? __ldg(src + 64) : z;
    double acc = 0.0;
    auto step = [&](int x) {
        // both bits are the same in every lane of a column: warp-uniform branches
        if (!(x & FOLD_SKIP)) acc += term(x & FOLD_MASK);
        if (x & FOLD_FLAG) {
            if (r < nrow) store(r, ck, acc);
            acc = 0.0;
            ++k;
            r = 32 * fold_group(k, warp) + lane;
            ck = nk;
            nk = pre(32 * fold_group(k + 1, warp) + lane);
        }
    };
    for (int q = 0; q < nq; ++q) {
        const int4 e = e0;
        e0 = e1;
        e1 = e2;
        e2 = q + 3 < nq ? __ldg(src + 32 * (q + 3)) : z;
        step(e.x);
        step(e.y);
        step(e.z);
        step(e.w);
    }
}

// One CTA per primitive pair, solid-harmonic rows:
//   H[m_a m_b][p] = sign(p) * sum_a (pref C_a[m_a][a]) sum_b C_b[m_b][b] E_ab^p
// by the factorised fold (one Cartesian index at a time, structural zeros skipped; the row
// streams and the G recipes are built on the host).  G of m_b = 0 is made first; then per
// m_b: the Q stage (one FMA per entry from G), a barrier, the W stage and G of m_b + 1 (G of
// m_b is no longer read), a barrier, then the H stage of m_b together with the Q stage of
// m_b + 1 (which touch disjoint arrays), a barrier.  On the split path the H stage also keeps
// each column's largest exponent, and the column scales are written at the end.
template <bool SCALES>  // the split path: pairs carry column scales (cs_off >= 0)
__global__ void __launch_bounds__(PAIR_SOLID_THREADS, 2) pair_h_solid_kernel(
    const DPair* __restrict__ pairs, const WorkItem* __restrict__ items, const DShell* __restrict__ sh,
    const double* __restrict__ exps, const double* __restrict__ ncoef, double* __restrict__ ws,
    double* __restrict__ ws_info, int lcap, int qcap, int wcap, int gcap, unsigned* status) {
    extern __shared__ double fold_smem[];
    const int etab = etab_of(lcap), ccap = ncoef_of(lcap) + 1;
    double* E = fold_smem;        // 3 etab
    double* Csa = E + 3 * etab;   // ccap: C_a, then a zero at ncoef(la)
    double* Csb = Csa + ccap;     // ccap: C_b, then a zero at ncoef(lb)
    double* Q = Csb + ccap;       // qcap (>= maxq + 1 of this pair's tables); Q[maxq] zero
    double* W = Q + qcap;         // wcap
    double* G = W + wcap;         // gcap (>= maxg + 1): the m_b's C_b E^z products, then a zero
    int* cexp = reinterpret_cast<int*>(G + gcap);  // pyr(2 lcap): largest exponent field per column
    __shared__ double s_pref;
    const WorkItem it = items[blockIdx.x];
    const DPair pr = pairs[it.q];
    const bool scales = SCALES && pr.cs_off >= 0;
    if (SCALES)
        for (int p = threadIdx.x; p < pr.np; p += blockDim.x) cexp[p] = 0;  // ordered by pair_setup's barriers
    const int la = sh[pr.sa].l, lb = sh[pr.sb].l;
    const int kp = it.a;
    const int nca = ncart(la), ncb = ncart(lb), nsb = 2 * lb + 1;
    for (int i = threadIdx.x; i < (2 * la + 1) * nca; i += blockDim.x) Csa[i] = c_solid[c_solid_off[la] + i];
    for (int i = threadIdx.x; i < nsb * ncb; i += blockDim.x) Csb[i] = c_solid[c_solid_off[lb] + i];
    if (threadIdx.x == 0) {
        Csa[ncoef_of(la)] = 0.0;
        Csb[ncoef_of(lb)] = 0.0;
        Q[c_fold.pair[la][lb].maxq] = 0.0;
    }
    pair_setup(pr, kp, sh, exps, ncoef, ws_info, E, etab, &s_pref);
    // the prefactor rides on C_a (one multiply per coefficient instead of one per H entry);
    // each thread scales the entries it loaded, and the first read is two barriers away
    const double pref = s_pref;
    for (int i = threadIdx.x; i < (2 * la + 1) * nca; i += blockDim.x) Csa[i] *= pref;

    const int np = pr.np;
    const int64_t ldh = (int64_t)pr.Kab * np;
    double* H = ws + pr.h_off + (int64_t)kp * np;
    const double* Ex = E;
    const double* Ey = E + etab;
    const double* Ez = E + 2 * etab;
    const FoldPairTab tab = c_fold.pair[la][lb];
    const FoldSeg* segs = c_fold.segs + tab.seg0;
    const int* __restrict__ h_out = c_fold.h_out;
    const int hrows = (2 * la + 1) * np;
    const bool sign = pr.sign;

    // G of one m_b: C_b[m_b][b] E^z_{az bz v} once per (b, az, v), so that a Q entry is one FMA
    auto g_build = [=](const FoldSeg* sg) {
        const int* rec = c_fold.g_rec + sg->g_off;
        for (int g = threadIdx.x; g < sg->g_n; g += blockDim.x) {
            const int r = __ldg(&rec[g]);
            G[g] = Csb[r & 1023] * Ez[r >> 10];
        }
        if (threadIdx.x == 0) G[sg->g_n] = 0.0;
    };
    auto q_term = [=](int x) { return G[x & 1023] * Ey[x >> 10]; };
    auto no_pre = [](int) { return 0; };
    auto q_store = [=](int r, int, double v) { Q[r] = v; };
    g_build(segs);
    __syncthreads();
    fold_stage(segs[0].q_ws, segs[0].q_nrow, c_fold.q_ent, q_term, no_pre, q_store);
    __syncthreads();
    for (int mb = 0; mb < nsb; ++mb) {
        const FoldSeg* sg = segs + mb;
        fold_stage(sg->w_ws, sg->w_nrow, c_fold.w_ent, [=](int x) { return Ex[x & 1023] * Q[x >> 10]; }, no_pre,
                   [=](int r, int, double v) { W[r] = v; });
        if (mb + 1 < nsb) g_build(sg + 1);  // G of m_b is done with: the next Q stage follows the barrier
        __syncthreads();
        const int h_row0 = sg->h_row0;
        fold_stage(sg->h_ws, hrows, c_fold.h_ent, [=](int x) { return Csa[x & 1023] * W[x >> 10]; },
                   [=](int r) { return r < hrows ? __ldg(&h_out[h_row0 + r]) : 0; },
                   [=](int, int o, double v) {
                       const int ma = o & 15, p = (o >> 4) & 0xffff;
                       const bool neg = sign && ((o >> 30) & 1);
                       if (scales) atomicMax(&cexp[p], exp_field_of(v));
                       // the sign as a bit flip, off the FP64 pipe
                       H[(int64_t)(ma * nsb + mb) * ldh + p] =
                           __longlong_as_double(__double_as_longlong(v) ^ ((long long)neg << 63));
                   });
        if (mb + 1 < nsb) fold_stage(sg[1].q_ws, sg[1].q_nrow, c_fold.q_ent, q_term, no_pre, q_store);
        __syncthreads();
    }
    if (scales)
        write_col_scales(cexp, np, reinterpret_cast<int*>(reinterpret_cast<char*>(ws) + pr.cs_off) + (int64_t)kp * np);
}

}  // namespace

cudaError_t init_prep_tables(const double* host_coefs, const int* host_tuv, const void* host_fold) {
    int off[LMAX + 2];
    off[0] = 0;
    for (int l = 0; l <= LMAX; ++l) off[l + 1] = off[l] + (2 * l + 1) * ncart(l);
    if (off[LMAX + 1] != NSOLID_PACKED) return cudaErrorInvalidValue;
    cudaError_t e = cudaMemcpyToSymbol(c_solid, host_coefs, sizeof(double) * NSOLID_PACKED);
    if (e != cudaSuccess) return e;
    e = cudaMemcpyToSymbol(c_solid_off, off, sizeof(off));
    if (e != cudaSuccess) return e;
    // fold lists: device copies held for the life of the process (one set per device)
    const FoldHost& F = *static_cast<const FoldHost*>(host_fold);
    FoldDev d{};
    const std::vector<int>* src[6] = {&F.q_ent, &F.w_ent, &F.h_ent, &F.h_out, &F.wstart, &F.g_rec};
    const int** dst[6] = {&d.q_ent, &d.w_ent, &d.h_ent, &d.h_out, &d.wstart, &d.g_rec};
    for (int k = 0; k < 6; ++k) {
        int* p = nullptr;
        const size_t bytes = sizeof(int) * (src[k]->size() + 1);
        if ((e = cudaMalloc(&p, bytes)) != cudaSuccess) return e;
        if ((e = cudaMemcpy(p, src[k]->data(), sizeof(int) * src[k]->size(), cudaMemcpyHostToDevice)) != cudaSuccess)
            return e;
        *dst[k] = p;
    }
    FoldSeg* segs = nullptr;
    if ((e = cudaMalloc(&segs, sizeof(FoldSeg) * F.segs.size())) != cudaSuccess) return e;
    if ((e = cudaMemcpy(segs, F.segs.data(), sizeof(FoldSeg) * F.segs.size(), cudaMemcpyHostToDevice)) !=
        cudaSuccess)
        return e;
    d.segs = segs;
    for (int a = 0; a <= LMAX; ++a)
        for (int b = 0; b <= LMAX; ++b) d.pair[a][b] = F.pair[a][b];
    if ((e = cudaMemcpyToSymbol(c_fold, &d, sizeof(d))) != cudaSuccess) return e;
    int qmax = 0, wmax = 0, gmax = 0;
    for (int a = 0; a <= LMAX; ++a)
        for (int b = 0; b <= LMAX; ++b) {
            qmax = std::max(qmax, F.pair[a][b].maxq + 1);
            wmax = std::max(wmax, F.pair[a][b].maxw);
            gmax = std::max(gmax, F.pair[a][b].maxg + 1);
        }
    for (const void* k : {(const void*)pair_h_solid_kernel<false>, (const void*)pair_h_solid_kernel<true>})
        if ((e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)fold_smem_bytes(LMAX, qmax, wmax, gmax))) != cudaSuccess)
            return e;
    return cudaMemcpyToSymbol(g_tuv_prep, host_tuv, sizeof(int) * NHERM_TOT);
}

cudaError_t launch_norm(const DShell* sh, int nshell, const double* exps, const double* coefs, double* ncoef,
                        unsigned* status, cudaStream_t st) {
    if (nshell <= 0) return cudaSuccess;
    norm_kernel<<<(nshell + 127) / 128, 128, 0, st>>>(sh, nshell, exps, coefs, ncoef, status);
    return cudaGetLastError();
}

cudaError_t launch_pair_h(const DPair* pairs, const WorkItem* items, int nitems, const DShell* sh,
                          const double* exps, const double* ncoef, double* ws, double* ws_info, bool solid, bool scales,
                          int fold_lcap, int fold_qcap, int fold_wcap, int fold_gcap, unsigned* status,
                          cudaStream_t st) {
    if (nitems <= 0) return cudaSuccess;
    if (solid) {
        if (fold_lcap < 0 || fold_lcap > LMAX) return cudaErrorInvalidValue;
        const size_t smem = fold_smem_bytes(fold_lcap, fold_qcap, fold_wcap, fold_gcap);
        if (scales)
            pair_h_solid_kernel<true><<<nitems, PAIR_SOLID_THREADS, smem, st>>>(
                pairs, items, sh, exps, ncoef, ws, ws_info, fold_lcap, fold_qcap, fold_wcap, fold_gcap, status);
        else
            pair_h_solid_kernel<false><<<nitems, PAIR_SOLID_THREADS, smem, st>>>(
                pairs, items, sh, exps, ncoef, ws, ws_info, fold_lcap, fold_qcap, fold_wcap, fold_gcap, status);
    } else
        pair_h_kernel<<<nitems, PAIR_THREADS, 0, st>>>(pairs, items, sh, exps, ncoef, ws, ws_info, status);
    return cudaGetLastError();
}

}  // namespace lx
