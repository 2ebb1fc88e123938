// Internal declarations shared by the library's translation units (not part of the ABI).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "lx_eri.h"

namespace lx {

constexpr int LMAX = LX_LMAX;                       // largest shell l
constexpr int LTOT = 4 * LMAX;                      // largest total L of a quartet (28)
constexpr int NCART_MAX = (LMAX + 1) * (LMAX + 2) / 2;  // 36
constexpr int NSOL_MAX = 2 * LMAX + 1;              // 15
constexpr int NHERM_TOT = (LTOT + 1) * (LTOT + 2) * (LTOT + 3) / 6;  // pyr(28) = 4495
constexpr int NHERM_PAIR = (2 * LMAX + 1) * (2 * LMAX + 2) * (2 * LMAX + 3) / 6;  // pyr(14) = 680: Hermite indices of one pair

// Boys table: F_n(T_k), n = 0..BOYS_NROW-1, T_k = k * BOYS_DT for k = 0..BOYS_NPT-1.
// Taylor expansion of order BOYS_ORDER-1 around the nearest grid point covers T < BOYS_TMAX.
constexpr int BOYS_ORDER = 8;
constexpr int BOYS_NROW = LTOT + BOYS_ORDER;        // 36
constexpr int BOYS_NPT = 361;
constexpr double BOYS_DT = 0.1;
constexpr double BOYS_TMAX = 36.0;

__host__ __device__ inline int pyr(int n) { return (n + 1) * (n + 2) * (n + 3) / 6; }
__host__ __device__ inline int ncart(int l) { return (l + 1) * (l + 2) / 2; }
__host__ __device__ inline int nfun(int l, bool solid) { return solid ? 2 * l + 1 : (l + 1) * (l + 2) / 2; }
// Pyramidal ordinal of a Hermite triplet (t,u,v): lower totals first; within total n,
// i = u+v ascending, then v ascending.  Within one total this is the Cartesian order.
__host__ __device__ inline int hidx(int t, int u, int v) {
    int n = t + u + v, i = u + v;
    return n * (n + 1) * (n + 2) / 6 + i * (i + 1) / 2 + v;
}

// Device status word bits (see lx_eri_sync_status).
enum : unsigned { ST_BAD_INDEX = 1u, ST_BAD_INPUT = 2u, ST_TIMEOUT = 4u };

struct DShell {  // 48 bytes
    int l, K, prim_off;
    int bf;  // first basis function of the shell (J/K digestion)
    double A[3];
    double pad2;
};

struct DPair {  // one shell pair on one side of the quartet
    int sa, sb;     // shells
    int Kab;        // K_a * K_b primitive pairs
    int nrow;       // nfun(l_a) nfun(l_b)
    int np;         // pyr(l_a + l_b)
    int sign;       // 1: ket side, columns carry (-1)^{|p|}
    int solid;      // 1: solid-harmonic rows
    int pad;
    int64_t h_off;     // H block (doubles): [nrow][Kab*np]
    int64_t info_off;  // pair scalars (doubles): [Kab][4] = zeta_p, P
    // split path: column scales of H, int[Kab*np] at this many bytes from the workspace base
    // (c_k with |H[.][k]| < 2^c_k over the column, 0 for a zero column), written by the pair's
    // H kernel; -1: none
    int64_t cs_off;
};

struct DQuartet {
    int pb, pk;          // bra / ket pair ids
    int L, np, nq;       // L = l_bra + l_ket, Hermite counts
    int nab, ncd;        // output rows / columns
    int kbra, kket;      // primitive-pair counts
    int nr;              // pyr(L)
    int64_t rr_off;      // [kbra][kket][nr] doubles
    int64_t x_off;       // [nab][kket*nq] doubles
    int64_t out_off;     // output block in the caller's buffer (J/K digestion: in the workspace)
};

struct WorkItem {  // generic work descriptor: owner + two tile indices
    int q, a, b, c;
};

// ----------------------------------------------------------------- per-TU launchers
// Tables (called once per device with that device current).
cudaError_t init_boys_table(const double* host_table);      // lx_boys_r.cu
cudaError_t init_prep_tables(const double* host_coefs, const int* host_tuv,
                             const void* host_fold);  // lx_prep.cu (host_fold: const FoldHost*)
cudaError_t init_tuv_table(const int* host_tuv);           // lx_gemm.cu

cudaError_t launch_norm(const DShell* sh, int nshell, const double* exps, const double* coefs, double* ncoef,
                        unsigned* status, cudaStream_t st);
// H blocks at ws + h_off, pair scalars at ws_info + info_off.
cudaError_t launch_pair_h(const DPair* pairs, const WorkItem* items, int nitems, const DShell* sh,
                          const double* exps, const double* ncoef, double* ws, double* ws_info, bool solid,
                          bool scales, int fold_lcap, int fold_qcap, int fold_wcap, int fold_gcap,
                          unsigned* status, cudaStream_t st);  // scales: pairs carry cs_off; solid fold:
                                                               // largest l, Q, W and G capacities
// J/K digestion of the blocks at ws + out_off, one CTA per quartet (lx_jk.cu).  J or K may
// be null.
cudaError_t launch_jk_digest(const DQuartet* qd, const DPair* pairs, const DShell* sh, int nquartet,
                             const double* ws, bool solid, const double* D, int64_t nbf, double* J, double* K,
                             cudaStream_t st);
// J/K straight from X = [ab|q] and the ket H, one CTA per quartet walking K_ket N_q in
// chunks of qc columns (lx_jk.cu); smem = jk_direct_smem(...) over the chunk's quartets.
constexpr size_t JKD_SMEM_MAX = 200 * 1024;
size_t jk_direct_smem(int nab, int ncd, int nb, int nc, int nd, int qc);
cudaError_t launch_jk_direct(const DQuartet* qd, const DPair* pairs, const DShell* sh, int nquartet, int qc,
                             size_t smem, const double* ws, bool solid, const double* D, int64_t nbf, double* J,
                             double* K, cudaStream_t st);
cudaError_t init_jk_kernels();
cudaError_t launch_boys_r(const DQuartet* qd, const DPair* pairs, const WorkItem* items, int nitems, int lmax,
                          double* ws, unsigned* status, cudaStream_t st);  // lmax: largest L of the items
// items grouped by tile shape: counts[v] items of shape v, in shape order; counters[v] is the
// zero-initialised work counter of shape v's launch
cudaError_t launch_gemm1(const DQuartet* qd, const DPair* pairs, const WorkItem* items, const int* counts, double* ws,
                         int* counters, unsigned* status, cudaStream_t st);
cudaError_t launch_gemm2(const DQuartet* qd, const DPair* pairs, const WorkItem* items, const int* counts,
                         const double* ws_in, double* out, int* counters, unsigned* status, cudaStream_t st);
cudaError_t launch_boys(int mmax, const double* T, int64_t n, double* F, unsigned* status, cudaStream_t st);
cudaError_t launch_hermite_r(int L, const double* params, int64_t n, double* R, unsigned* status, cudaStream_t st);

// Router (lx_router.cu).
cudaError_t init_router_kernels();
cudaError_t launch_features(const DShell* sh, const double* exps, const int* q4, int64_t nq, float* feat,
                            cudaStream_t st);
cudaError_t launch_mlp_forward(const void* p16, const float* feat, int64_t n, float* out, cudaStream_t st);
cudaError_t launch_mlp_grad(const float* params, const float* feat, const float* target, int64_t n, float* grad,
                            float* loss, cudaStream_t st);
cudaError_t launch_mlp_adam(float* params, float* m, float* v, float* grad, void* p16, int step, float lr, float b1,
                            float b2, float eps, cudaStream_t st);

// FP64 GEMM tile shapes (shared by the planner, the autotuner and the kernels).
enum : int { GEMM_V32x64 = 0, GEMM_V64x32 = 1, GEMM_V32x32 = 2, GEMM_V64x64 = 3, GEMM_NVARIANT = 4 };
__host__ __device__ inline int gemm_bm(int v) { return (v == GEMM_V64x32 || v == GEMM_V64x64) ? 64 : 32; }
__host__ __device__ inline int gemm_bn(int v) { return (v == GEMM_V32x64 || v == GEMM_V64x64) ? 64 : 32; }
constexpr int GEMM_BK = 16;

// Real solid harmonics have fixed parities of the x, y, z exponents, so the matrix C of one
// shell is block diagonal over the (at most 4) parity classes of its Cartesian components.

// Factorised solid fold of one primitive pair (la, lb), per solid function m_b of b:
//   G[b az v]         = C_b[m_b][bx by bz] E^z_{az bz v}                          (nonzero C_b only)
//   Q[ay az bx u v]   = sum_by G[b az v] E^y_{ay by u}                             (bz = lb - bx - by)
//   W[a u v t]        = sum_bx E^x_{ax bx t} Q[ay az bx u v]
//   H[m_a m_b][t u v] = sum_a C_a[m_a][a] W[a t u v]
// Only entries that can be nonzero (t <= ax + bx, u <= ay + by, v <= az + bz, nonzero C) are
// kept.  Each stage's rows are sorted by length and taken in groups of 32 (lane i of a warp
// owns row 32 g + i); every row of a group is padded to the group's longest row with null
// entries that multiply by an explicit zero, and a group of empty rows gets one null entry.
// Warp w takes groups fold_group(k, w) for k = 0, 1, ...: round k of FOLD_NWARP groups is
// dealt to the warps in order for even k and in reverse for odd k, which evens out the warps'
// work on groups sorted by length.  Each warp reads one stream: its groups in order, column j of a group (entry j
// of its 32 rows) after column j - 1.  Every entry of a group's last column carries
// FOLD_FLAG (end of those rows: store them and move to the warp's next group), and every
// entry of a column with no real entry carries FOLD_SKIP (nothing to add).  Columns are stored
// four at a time, lane-major: entry j of lane i's current row at stream + 128 (j / 4) + 4 i +
// j % 4, so one 16-byte load per lane fetches four; a stream is padded to whole quads with
// skipped null columns.  Warp w's stream of a stage is ent[ws[w] .. ws[w + 1]) (ws = wstart +
// the stage's offset, FOLD_NWARP + 1 bounds).
//   G recipe (g_rec[g_off + g]): coefficient index (m_b ncart(lb) + b) | E^z index << 10
//   Q entry: G index | E^y index << 10
//   W entry: E^x index | Q row << 10
//   H entry: coefficient index (m_a ncart(la) + a) | W row << 10;
//   h_out[row] = m_a | p << 4 | (t + u + v odd) << 30, with p = hidx(t, u, v)
// E^d index = (i (lb+1) + j) (la+lb+1) + t for exponents (i, j) on a and b.  Null entries
// multiply by a zero: G index g_n in a Q row (the zero after the m_b's G entries), coefficient
// index (2la+1) ncart(la) in an H row (one past the shell's coefficients), Q row maxq of the
// (la, lb) (the row after its largest Q stage) in a W row.
constexpr int FOLD_NWARP = 16;              // warps of the fold kernel (one stream each)
constexpr int FOLD_FLAG = INT32_MIN;          // bit 31: the last column of a group
constexpr int FOLD_SKIP = 1 << 30;            // bit 30: a column of null entries only
constexpr int FOLD_MASK = FOLD_SKIP - 1;      // the entry itself
// Group of round k of warp w.
__host__ __device__ inline int fold_group(int k, int w) {
    return k * FOLD_NWARP + ((k & 1) ? FOLD_NWARP - 1 - w : w);
}
constexpr int FOLD_QMAX = 8191;   // bound on the Q rows of one m_b (5688 at la = lb = 7)
constexpr int FOLD_WMAX = 16383;  // bound on the W rows of one m_b (13542 at la = lb = 7)
constexpr int FOLD_GMAX = 1023;   // bound on the G entries of one m_b (600 at la = lb = 7)
constexpr int FOLD_CMAX = NSOL_MAX * NCART_MAX;  // coefficients of one shell (540 at l = 7)
static_assert(FOLD_CMAX < 1024 && (LMAX + 1) * (LMAX + 1) * (2 * LMAX + 1) <= 1024, "fold entry fields of 10 bits");
struct FoldSeg {
    int q_ws, q_nrow, w_ws, w_nrow, h_ws, h_row0;  // each stage's offset in wstart; h_out offset
    int g_off, g_n;                                 // the m_b's G recipes in g_rec
};
struct FoldPairTab {
    int seg0;  // segments seg0 .. seg0 + 2 lb (one per m_b)
    int maxq, maxw;  // largest Q and W row counts over the m_b (Q row maxq is the zero row)
    int maxg;        // largest G count over the m_b
};
constexpr int NSOLID_PACKED = [] {
    int n = 0;
    for (int l = 0; l <= LMAX; ++l) n += (2 * l + 1) * ((l + 1) * (l + 2) / 2);
    return n;
}();  // solid-harmonic coefficients of l = 0..LMAX, packed

// lx_eri_batch with the descriptors uploaded from pageable memory, allocating nothing
// (lx_api.cu; used by lx_eri_batch_static).
int eri_batch_unstaged(const lx_shell* shells, int32_t nshell, const double* exps, const double* coefs,
                       int32_t nprim_total, const lx_quartet* quartets, int64_t nquartet, int32_t flags, double* out,
                       void* workspace, size_t workspace_bytes, void* cuda_stream);

// Entry-point preamble (lx_api.cu): refuses a capturing stream (LX_ERR_CUDA, with `who` in
// lx_last_cuda_error), then sets up the current device (architecture check, tables).
int entry_prepare(void* cuda_stream, const char* who, unsigned** status);
// LX_ERR_CUDA, with the error's text kept for lx_last_cuda_error.
int report_cuda_error(cudaError_t e);

// Host-side table generators (lx_tables.cpp).
void make_boys_table(double* table);        // BOYS_NROW * BOYS_NPT
void make_solid_coefs(double* coefs);       // packed: l = 0..LMAX, (2l+1) x ncart(l) each
int solid_offset(int l);                    // offset of shell l's block in the packed array
void make_tuv_table(int* tuv);              // NHERM_TOT entries: t | u << 8 | v << 16
}  // namespace lx

#include <vector>
namespace lx {
struct FoldHost {
    std::vector<int> q_ent, w_ent, h_ent, h_out, wstart, g_rec;
    std::vector<FoldSeg> segs;
    FoldPairTab pair[LMAX + 1][LMAX + 1];
};
// Compressed fold lists for every (la, lb); false if a count exceeds FOLD_QMAX / FOLD_WMAX.
bool make_fold_lists(const double* coefs, FoldHost& F);
// The fold tables built once for this process (valid after the first device set-up).
const FoldHost* fold_tables();

}  // namespace lx
