// C ABI of the library: input validation, batch planning and the launch sequence of the
// matrix form of MD4 (paper, Section 2, pseudocode "md4"; Section 3):
//   norm    -> normalised contraction coefficients
//   pair_h  -> per primitive pair: zeta_p, P and the H matrix (E recursions, solid fold)
//   boys_r  -> per primitive quartet: Boys function and [r]^(0) by Eq. md1
//   gemm1   -> [ab|q] = H_ab [p|q]                                  (Eq. make-abq)
//   gemm2   -> (ab|cd) = [ab|q] H_cd^T                              (Eq. make-abcd)
// The host side only validates, deduplicates shell pairs, lays out the caller's workspace
// and builds work lists; every arithmetic step of the method runs in the kernels.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <map>
#include <mutex>
#include <unordered_map>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "lx_internal.cuh"
#include "lx_split.cuh"

namespace lx {
namespace {

__device__ unsigned g_status_word;

constexpr int MAX_DEVICES = 64;
// Planner flag of lx_eri_jk (never accepted from callers): each quartet's block goes to the
// workspace and is digested into J and K there.
constexpr int32_t JK_DIGEST = 0x40000000;
std::mutex g_init_mutex;
bool g_dev_ready[MAX_DEVICES];
unsigned* g_status_ptr[MAX_DEVICES];

thread_local char t_cuda_msg[256] = "no error";

// Stage timing (LX_TIME_STAGES): events recorded around each stage, read back by
// lx_eri_stage_times.
struct PendingTiming {
    cudaStream_t stream;
    cudaEvent_t begin, end;
    int stage;
    int launches;
};
std::mutex g_timing_mutex;
std::vector<PendingTiming> g_pending;

struct StageTimer {
    bool on;
    cudaStream_t st;
    cudaEvent_t cur = nullptr;
    cudaError_t begin() {
        if (!on) return cudaSuccess;
        cudaError_t e = cudaEventCreate(&cur);
        if (e != cudaSuccess) return e;
        return cudaEventRecord(cur, st);
    }
    cudaError_t end(int stage, int launches) {
        if (!on) return cudaSuccess;
        cudaEvent_t e1;
        cudaError_t e = cudaEventCreate(&e1);
        if (e != cudaSuccess) return e;
        if ((e = cudaEventRecord(e1, st)) != cudaSuccess) return e;
        std::lock_guard<std::mutex> lock(g_timing_mutex);
        g_pending.push_back({st, cur, e1, stage, launches});
        cur = nullptr;
        return cudaSuccess;
    }
};

int cuda_fail(cudaError_t e) {
    std::snprintf(t_cuda_msg, sizeof(t_cuda_msg), "%s: %s", cudaGetErrorName(e), cudaGetErrorString(e));
    return LX_ERR_CUDA;
}

FoldHost g_fold;  // the solid fold's row lists (host copy), built with the first device
bool g_fold_ready = false;

// Once per device, with that device current: check the architecture, upload the tables,
// look up the status word.  Returns LX_OK or an error code; *status receives the word.
int ensure_device(unsigned** status) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e);
    if (dev < 0 || dev >= MAX_DEVICES) return LX_ERR_ARCH;
    std::lock_guard<std::mutex> lock(g_init_mutex);
    if (!g_dev_ready[dev]) {
        int major = 0, minor = 0;
        e = cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
        if (e != cudaSuccess) return cuda_fail(e);
        e = cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
        if (e != cudaSuccess) return cuda_fail(e);
        if (major != 10 || minor != 3) return LX_ERR_ARCH;
        std::vector<double> boys(BOYS_NROW * BOYS_NPT);
        make_boys_table(boys.data());
        std::vector<double> solid(NSOLID_PACKED);
        make_solid_coefs(solid.data());
        std::vector<int> tuv(NHERM_TOT);
        make_tuv_table(tuv.data());
        if ((e = init_boys_table(boys.data())) != cudaSuccess) return cuda_fail(e);
        if (!g_fold_ready) {  // identical for every device; built once
            if (!make_fold_lists(solid.data(), g_fold)) return LX_ERR_SIZE;
            g_fold_ready = true;
        }
        if ((e = init_prep_tables(solid.data(), tuv.data(), &g_fold)) != cudaSuccess) return cuda_fail(e);
        if ((e = init_tuv_table(tuv.data())) != cudaSuccess) return cuda_fail(e);
        if ((e = init_split_kernels(tuv.data())) != cudaSuccess) return cuda_fail(e);
        if ((e = init_jk_kernels()) != cudaSuccess) return cuda_fail(e);
        if ((e = init_router_kernels()) != cudaSuccess) return cuda_fail(e);
        void* p = nullptr;
        if ((e = cudaGetSymbolAddress(&p, g_status_word)) != cudaSuccess) return cuda_fail(e);
        const unsigned zero = 0;
        if ((e = cudaMemcpyToSymbol(g_status_word, &zero, sizeof(zero))) != cudaSuccess) return cuda_fail(e);
        g_status_ptr[dev] = static_cast<unsigned*>(p);
        g_dev_ready[dev] = true;
    }
    *status = g_status_ptr[dev];
    return LX_OK;
}

inline size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

struct QuartetShape {
    int la, lb, lc, ld, Ka, Kb, Kc, Kd;
};

int validate(const lx_shell* shells, int32_t nshell, const double* exps, const double* coefs, int32_t nprim_total,
             const lx_quartet* quartets, int64_t nquartet, int32_t flags, bool need_prims) {
    if (nshell < 0 || nquartet < 0 || nprim_total < 0) return LX_ERR_SIZE;
    if ((nshell > 0 && !shells) || (nquartet > 0 && !quartets)) return LX_ERR_NULL;
    if (need_prims && nprim_total > 0 && (!exps || !coefs)) return LX_ERR_NULL;
    if (flags & ~(LX_SOLID | LX_PATH_SPLIT | LX_PATH_ROUTED | LX_TIME_STAGES | LX_SPLIT_DIGITS_MASK)) return LX_ERR_FLAGS;
    if ((flags & LX_PATH_ROUTED) && (flags & LX_PATH_SPLIT)) return LX_ERR_FLAGS;
    if (flags & LX_SPLIT_DIGITS_MASK) {  // a digit count: 4, 5 or 6, with the split path only
        const int nd = (flags & LX_SPLIT_DIGITS_MASK) >> 4;
        if (!(flags & LX_PATH_SPLIT) || nd < SPLIT_MIN_DIGITS || nd > SPLIT_NSLICE) return LX_ERR_FLAGS;
    }
    for (int32_t s = 0; s < nshell; ++s) {
        const lx_shell& d = shells[s];
        if (d.l < 0 || d.l > LX_LMAX || d.nprim < 1 || d.nprim > LX_KMAX || d.reserved != 0) return LX_ERR_SHELL;
        if (!std::isfinite(d.center[0]) || !std::isfinite(d.center[1]) || !std::isfinite(d.center[2]))
            return LX_ERR_SHELL;
        if (need_prims) {
            if (d.prim_offset < 0 || (int64_t)d.prim_offset + d.nprim > nprim_total) return LX_ERR_SHELL;
            for (int k = 0; k < d.nprim; ++k) {
                const double z = exps[d.prim_offset + k], c = coefs[d.prim_offset + k];
                if (!(std::isfinite(z) && z > 0.0) || !std::isfinite(c)) return LX_ERR_PRIMITIVE;
            }
        }
    }
    for (int64_t q = 0; q < nquartet; ++q) {
        for (int k = 0; k < 4; ++k)
            if (quartets[q].s[k] < 0 || quartets[q].s[k] >= nshell) return LX_ERR_QUARTET;
        if (quartets[q].out_offset < 0) return LX_ERR_QUARTET;
    }
    return LX_OK;
}

// ------------------------------------------------------------------ tuning table

// Tile shape per (class, contraction) of the FP64 GEMMs, filled by lx_eri_autotune or
// lx_tune_import; keys not in the table use GEMM_V32x64.
struct TuneKey {
    int la, lb, lc, ld, kbra, kket, solid;
    bool operator<(const TuneKey& o) const {
        const int a[7] = {la, lb, lc, ld, kbra, kket, solid}, b[7] = {o.la, o.lb, o.lc, o.ld, o.kbra, o.kket, o.solid};
        for (int i = 0; i < 7; ++i)
            if (a[i] != b[i]) return a[i] < b[i];
        return false;
    }
};
struct TuneVal {
    int v1, v2;
};
std::mutex g_tune_mutex;
std::map<TuneKey, TuneVal> g_tune;

TuneKey tune_key(const lx_shell* sh, const lx_quartet& q, bool solid) {
    return TuneKey{sh[q.s[0]].l, sh[q.s[1]].l, sh[q.s[2]].l, sh[q.s[3]].l, sh[q.s[0]].nprim * sh[q.s[1]].nprim,
                   sh[q.s[2]].nprim * sh[q.s[3]].nprim, solid ? 1 : 0};
}

// Forced tile shapes (autotuning); -1 = use the table.
struct Overrides {
    int v1 = -1, v2 = -1;
};

// ------------------------------------------------------------------ planning

struct PairKey {
    int64_t v;
    bool operator==(const PairKey& o) const { return v == o.v; }
};
struct PairKeyHash {
    size_t operator()(const PairKey& k) const { return std::hash<int64_t>()(k.v); }
};

struct Chunk {
    int64_t q_begin = 0, q_end = 0;
};

// Workspace bytes of one quartet's own data (without its pairs), for path flags `flags`.
size_t quartet_bytes(const lx_shell* sh, const lx_quartet& q, int flags) {
    const bool solid = flags & LX_SOLID, split = flags & LX_PATH_SPLIT;
    const lx_shell &a = sh[q.s[0]], &b = sh[q.s[1]], &c = sh[q.s[2]], &d = sh[q.s[3]];
    const int L = a.l + b.l + c.l + d.l, np = pyr(a.l + b.l), nq = pyr(c.l + d.l);
    const int64_t kbra = (int64_t)a.nprim * b.nprim, kket = (int64_t)c.nprim * d.nprim;
    const int64_t nab = (int64_t)nfun(a.l, solid) * nfun(b.l, solid), ncd = (int64_t)nfun(c.l, solid) * nfun(d.l, solid);
    const int64_t n1 = kket * nq;
    int64_t items = kbra * kket;
    // + 256 bytes per data block: each block starts on a 256-byte boundary
    size_t bytes = sizeof(DQuartet) + 8 * (size_t)(kbra * kket * pyr(L) + nab * n1) + 512;
    // J/K: the split path digests each block from the workspace; the FP64 path contracts
    // [ab|q] directly and stores no block
    if ((flags & JK_DIGEST) && split) bytes += 8 * (size_t)(nab * ncd) + 256;
    if (!split) {
        // bound: the 32 x 32 tile gives the most work items
        items += ((nab + 31) / 32) * ((n1 + 31) / 32);
        items += ((nab + 31) / 32) * ((ncd + 31) / 32);
    } else {
        // [p|q]^T and X digit planes with their segment exponents; H's go with the pair (pair_bytes)
        const int k1 = (int)(kbra * np), k2 = (int)n1;
        const int ra1 = split_rowpad(k2, SPLIT_TA), ra2 = split_rowpad((int)nab, SPLIT_TA);
        items += (ra1 + ra2) / 8;
        items += (ra1 / SPLIT_TA) * ((nab + SPLIT_TB - 1) / SPLIT_TB);
        items += (ra2 / SPLIT_TA) * ((ncd + SPLIT_TB - 1) / SPLIT_TB);
        bytes += sizeof(SplitQuartet) + 2 * sizeof(SplitGemmDesc) + sizeof(SplitRowsDesc);
        bytes += (size_t)split_dig_bytes(k2, k1, SPLIT_TA) + (size_t)split_dig_bytes((int)nab, k2, SPLIT_TA);
        bytes += 4 * ((size_t)ra1 + (size_t)ra2 * split_nseg(split_nkb(k2))) + 4 * 256;
    }
    return bytes + items * sizeof(WorkItem);
}

size_t pair_bytes(const lx_shell* sh, int sa, int sb, int flags) {
    const bool solid = flags & LX_SOLID, split = flags & LX_PATH_SPLIT;
    const lx_shell &a = sh[sa], &b = sh[sb];
    const int64_t kab = (int64_t)a.nprim * b.nprim;
    const int64_t rows = (int64_t)nfun(a.l, solid) * nfun(b.l, solid);
    const int64_t k = kab * pyr(a.l + b.l);
    size_t bytes = sizeof(DPair) + kab * sizeof(WorkItem) + 8 * (size_t)(kab * 4 + rows * k) + 512;
    if (split) {
        // H's digit planes (rows padded to at most SPLIT_TB), row exponents, column scales
        const int rp = split_rowpad((int)rows, SPLIT_TB);
        bytes += sizeof(SplitRowsDesc) + (size_t)split_dig_bytes((int)rows, (int)k, SPLIT_TB);
        bytes += 4 * (size_t)(rp + k) + 3 * 256;
        bytes += sizeof(WorkItem) * (size_t)(rp / 8);
    }
    return bytes;
}

constexpr size_t CHUNK_SLACK = 32 * 256;  // alignment padding of the chunk's regions and the work counters

size_t head_bytes(int nshell, int nprim) {
    return align256(sizeof(DShell) * (size_t)nshell) + 3 * align256(sizeof(double) * (size_t)nprim);
}

// Greedy chunking of the quartet list so that each chunk fits `budget` bytes.
int plan_chunks(const lx_shell* sh, const lx_quartet* qs, int64_t nq, int flags, size_t budget,
                std::vector<Chunk>& chunks) {
    chunks.clear();
    std::unordered_map<PairKey, int, PairKeyHash> seen;
    size_t used = CHUNK_SLACK;
    Chunk cur;
    cur.q_begin = 0;
    for (int64_t i = 0; i < nq; ++i) {
        const lx_quartet& q = qs[i];
        size_t add = quartet_bytes(sh, q, flags);
        const PairKey kb{((int64_t)q.s[0] << 32 | (uint32_t)q.s[1]) * 2};
        const PairKey kk{((int64_t)q.s[2] << 32 | (uint32_t)q.s[3]) * 2 + 1};
        const bool nb = !seen.count(kb), nk = !seen.count(kk);
        if (nb) add += pair_bytes(sh, q.s[0], q.s[1], flags);
        if (nk && !(kk == kb)) add += pair_bytes(sh, q.s[2], q.s[3], flags);
        if (used + add > budget) {
            if (i == cur.q_begin) return LX_ERR_WORKSPACE;  // one quartet does not fit
            cur.q_end = i;
            chunks.push_back(cur);
            cur.q_begin = i;
            seen.clear();
            used = CHUNK_SLACK;
            --i;  // retry this quartet in the new chunk
            continue;
        }
        used += add;
        seen[kb] = 1;
        seen[kk] = 1;
    }
    cur.q_end = nq;
    if (nq > 0) chunks.push_back(cur);
    return LX_OK;
}

// Layout of one chunk inside the workspace, built on the host.
struct ChunkPlan {
    std::vector<DPair> pairs;
    std::vector<DQuartet> quartets;
    std::vector<WorkItem> items_h, items_br, items_g1, items_g2;
    int br_lmax = 0;  // largest L of the chunk's quartets
    int digits = 6;   // split path: BF16 digits kept per value (one count per batch)
    int fold_lcap = 0, fold_qcap = 0, fold_wcap = 0, fold_gcap = 0;  // solid fold: largest l, Q, W and G of the chunk's pairs
    int jkd_qc = 0;          // J/K on the FP64 path: chunk width of jk_direct_kernel
    size_t jkd_smem = 0;     // and its shared memory
    size_t off_pairs = 0, off_quartets = 0, off_h = 0, off_br = 0, off_g1 = 0, off_g2 = 0, off_data = 0;
    int g1_counts[GEMM_NVARIANT] = {0, 0, 0, 0}, g2_counts[GEMM_NVARIANT] = {0, 0, 0, 0};
    size_t off_counters = 0;  // 2 x GEMM_NVARIANT work counters, uploaded as zeros with the blob
    // split path: one split-row desc per pair (H) and per quartet (X); the column scales of H
    // come from the pair kernels
    std::vector<SplitRowsDesc> srd;
    std::vector<SplitQuartet> sq;
    std::vector<SplitGemmDesc> sg1, sg2;
    std::vector<WorkItem> items_sr, items_sB, items_sg1, items_sD, items_sg2;
    size_t off_srd = 0, off_sq = 0, off_sg1 = 0, off_sg2 = 0;
    size_t off_isr = 0, off_isB = 0, off_isg1 = 0, off_isD = 0, off_isg2 = 0;
    size_t total = 0;         // bytes from the chunk base
    std::vector<char> blob;   // descriptor bytes [0, off_data)
};

void build_chunk(const lx_shell* sh, const lx_quartet* qs, const Chunk& ch, int flags, size_t chunk_base,
                 ChunkPlan& P, const Overrides& ov = Overrides()) {
    const bool solid = flags & LX_SOLID, split = flags & LX_PATH_SPLIT, jk = flags & JK_DIGEST;
    const int nd_flag = (flags & LX_SPLIT_DIGITS_MASK) >> 4, nd = nd_flag ? nd_flag : SPLIT_NSLICE;
    P.digits = nd;
    P.pairs.clear();
    P.quartets.clear();
    P.items_h.clear();
    P.items_br.clear();
    P.br_lmax = 0;
    P.fold_lcap = P.fold_qcap = P.fold_wcap = P.fold_gcap = 0;
    P.jkd_qc = 0;
    P.jkd_smem = 0;
    P.items_g1.clear();
    P.items_g2.clear();
    P.srd.clear();
    P.sq.clear();
    P.sg1.clear();
    P.sg2.clear();
    for (auto* v : {&P.items_sr, &P.items_sB, &P.items_sg1, &P.items_sD, &P.items_sg2})
        v->clear();
    std::unordered_map<PairKey, int, PairKeyHash> pid;
    auto get_pair = [&](int sa, int sb, int side) {
        const PairKey k{((int64_t)sa << 32 | (uint32_t)sb) * 2 + side};
        auto f = pid.find(k);
        if (f != pid.end()) return f->second;
        DPair p{};
        p.cs_off = -1;  // set with the data layout on the split path
        p.sa = sa;
        p.sb = sb;
        p.Kab = sh[sa].nprim * sh[sb].nprim;
        p.nrow = nfun(sh[sa].l, solid) * nfun(sh[sb].l, solid);
        p.np = pyr(sh[sa].l + sh[sb].l);
        p.sign = side;
        p.solid = solid ? 1 : 0;
        const int id = (int)P.pairs.size();
        P.pairs.push_back(p);
        pid.emplace(k, id);
        return id;
    };
    for (int64_t i = ch.q_begin; i < ch.q_end; ++i) {
        const lx_quartet& q = qs[i];
        DQuartet d{};
        d.pb = get_pair(q.s[0], q.s[1], 0);
        d.pk = get_pair(q.s[2], q.s[3], 1);
        const lx_shell &a = sh[q.s[0]], &b = sh[q.s[1]], &c = sh[q.s[2]], &dd = sh[q.s[3]];
        d.L = a.l + b.l + c.l + dd.l;
        d.np = pyr(a.l + b.l);
        d.nq = pyr(c.l + dd.l);
        d.nab = nfun(a.l, solid) * nfun(b.l, solid);
        d.ncd = nfun(c.l, solid) * nfun(dd.l, solid);
        d.kbra = a.nprim * b.nprim;
        d.kket = c.nprim * dd.nprim;
        d.nr = pyr(d.L);
        d.out_off = q.out_offset;
        P.quartets.push_back(d);
    }
    // work lists
    for (int i = 0; i < (int)P.pairs.size(); ++i)
        for (int kp = 0; kp < P.pairs[i].Kab; ++kp) P.items_h.push_back({i, kp, 0, 0});
    if (solid && g_fold_ready)
        for (const DPair& pr : P.pairs) {
            const FoldPairTab& t = g_fold.pair[sh[pr.sa].l][sh[pr.sb].l];
            P.fold_lcap = std::max(P.fold_lcap, std::max(sh[pr.sa].l, sh[pr.sb].l));
            P.fold_qcap = std::max(P.fold_qcap, t.maxq + 1);
            P.fold_wcap = std::max(P.fold_wcap, t.maxw);
            P.fold_gcap = std::max(P.fold_gcap, t.maxg + 1);
        }
    std::vector<int64_t> cost1, cost2;
    {
        std::lock_guard<std::mutex> lock(g_tune_mutex);
        for (int i = 0; i < (int)P.quartets.size(); ++i) {
            const DQuartet& d = P.quartets[i];
            for (int k = 0; k < d.kbra * d.kket; ++k) P.items_br.push_back({i, k, 0, 0});
            P.br_lmax = std::max(P.br_lmax, d.L);
            if (split) continue;
            // untuned: 64-row tiles once the bra has 128 rows or more (measured on (ii|ii)),
            // 32-row tiles for smaller classes
            int v1 = d.nab >= 128 ? GEMM_V64x32 : GEMM_V32x64, v2 = v1;
            auto f = g_tune.find(tune_key(sh, qs[ch.q_begin + i], solid));
            if (f != g_tune.end()) {
                v1 = f->second.v1;
                v2 = f->second.v2;
            }
            if (ov.v1 >= 0) v1 = ov.v1;
            if (ov.v2 >= 0) v2 = ov.v2;
            const int n1 = d.kket * d.nq, k1 = d.kbra * d.np;
            const int mt1 = (d.nab + gemm_bm(v1) - 1) / gemm_bm(v1), nt1 = (n1 + gemm_bn(v1) - 1) / gemm_bn(v1);
            const int mt2 = (d.nab + gemm_bm(v2) - 1) / gemm_bm(v2), nt2 = (d.ncd + gemm_bn(v2) - 1) / gemm_bn(v2);
            for (int m = 0; m < mt1; ++m)
                for (int n = 0; n < nt1; ++n) {
                    P.items_g1.push_back({i, m, n, v1});
                    cost1.push_back((int64_t)gemm_bm(v1) * gemm_bn(v1) * k1);
                }
            if (jk) continue;  // J/K straight from [ab|q]: no second transform
            for (int m = 0; m < mt2; ++m)
                for (int n = 0; n < nt2; ++n) {
                    P.items_g2.push_back({i, m, n, v2});
                    cost2.push_back((int64_t)gemm_bm(v2) * gemm_bn(v2) * n1);
                }
        }
    }
    if (jk && !split) {
        // chunk width of jk_direct_kernel: the widest whose shared memory lets 2 CTAs share an
        // SM, else the widest that fits at all
        P.jkd_qc = 0;
        for (int pass = 0; pass < 2 && P.jkd_qc == 0; ++pass)
            for (int qc = 16; qc >= 1; qc /= 2) {
                size_t need = 0;
                for (int i = 0; i < (int)P.quartets.size(); ++i) {
                    const lx_quartet& qq = qs[ch.q_begin + i];
                    const int nb_ = nfun(sh[qq.s[1]].l, solid), nc_ = nfun(sh[qq.s[2]].l, solid),
                              nd_ = nfun(sh[qq.s[3]].l, solid);
                    need = std::max(need, jk_direct_smem(P.quartets[i].nab, P.quartets[i].ncd, nb_, nc_, nd_, qc));
                }
                if (need <= (pass == 0 ? (size_t)110 * 1024 : JKD_SMEM_MAX)) {
                    P.jkd_qc = qc;
                    P.jkd_smem = need;
                    break;
                }
            }
    }
    // grouped by tile shape (one persistent launch each), largest tiles first within a shape:
    // the persistent launches hand items out round-robin
    auto lpt = [](std::vector<WorkItem>& items, const std::vector<int64_t>& cost, int* counts) {
        std::vector<size_t> idx(items.size());
        for (size_t k = 0; k < idx.size(); ++k) idx[k] = k;
        std::stable_sort(idx.begin(), idx.end(), [&](size_t x, size_t y) {
            if (items[x].c != items[y].c) return items[x].c < items[y].c;
            return cost[x] > cost[y];
        });
        std::vector<WorkItem> sorted(items.size());
        for (int v = 0; v < GEMM_NVARIANT; ++v) counts[v] = 0;
        for (size_t k = 0; k < idx.size(); ++k) {
            sorted[k] = items[idx[k]];
            ++counts[sorted[k].c];
        }
        items.swap(sorted);
    };
    lpt(P.items_g1, cost1, P.g1_counts);
    lpt(P.items_g2, cost2, P.g2_counts);
    if (split) {
        // split descriptors and work lists (offsets filled in below, with the data layout).
        // H's column scales depend on H alone, so each pair's scales and digit planes are made
        // once per chunk and shared by its quartets: descriptor p (< npair) splits H of pair
        // p, descriptor npair + i splits X of quartet i.
        const int npair = (int)P.pairs.size();
        for (int p = 0; p < npair; ++p) {
            const DPair& pr = P.pairs[p];
            const int k = pr.Kab * pr.np, tb = split_tb(pr.nrow);
            // columns scaled into (-1, 1): one pass, e = 0 per row
            P.srd.push_back(SplitRowsDesc{0, 0, 0, 0, k, pr.nrow, k, tb, split_nkb(k), -1, 1, 0, nd, 0});
            // digit kernels: one item per 8 consecutive rows, up to nrow rounded to 8 (the GEMMs
            // drop the output columns of B rows past nrow, so the rest of the last row tile is
            // never written)
            for (int row = 0; row < split_rowpad(pr.nrow, 8); row += 8) P.items_sB.push_back({p, row, 0, 0});
        }
        for (int i = 0; i < (int)P.quartets.size(); ++i) {
            const DQuartet& d = P.quartets[i];
            const int k1 = d.kbra * d.np, k2 = d.kket * d.nq;
            SplitQuartet q{};
            q.nkb1 = split_nkb(k1);
            q.nkb2 = split_nkb(k2);
            q.nd = nd;
            const DPair &pb = P.pairs[d.pb], &pk = P.pairs[d.pk];
            q.gidx_off = gidx_offset(sh[pb.sa].l + sh[pb.sb].l, sh[pk.sa].l + sh[pk.sb].l);
            P.sq.push_back(q);
            const int tb1 = split_tb(d.nab), tb2 = split_tb(d.ncd);
            // A2: X, one exponent per row and segment (the rows up to nab rounded to 8 are used)
            P.srd.push_back(SplitRowsDesc{0, 0, 0, 0, k2, d.nab, k2, SPLIT_TA, q.nkb2, +1, 2, split_nseg(q.nkb2), nd, 0});
            for (int row = 0; row < split_rowpad(k2, 8); row += 8) P.items_sr.push_back({i, row, 0, 0});
            // X's digit planes only after GEMM1
            for (int row = 0; row < split_rowpad(d.nab, 8); row += 8) P.items_sD.push_back({npair + i, row, 0, 0});
            const int mt1 = split_rowpad(k2, SPLIT_TA) / SPLIT_TA, nt1 = (d.nab + tb1 - 1) / tb1;
            const int mt2 = split_rowpad(d.nab, SPLIT_TA) / SPLIT_TA, nt2 = (d.ncd + tb2 - 1) / tb2;
            for (int m = 0; m < mt1; ++m)
                for (int n = 0; n < nt1; ++n) P.items_sg1.push_back({i, m, n, 0});
            for (int m = 0; m < mt2; ++m)
                for (int n = 0; n < nt2; ++n) P.items_sg2.push_back({i, m, n, 0});
        }
        // the persistent split GEMM hands items to CTAs in a fixed stride: longest first
        std::stable_sort(P.items_sg1.begin(), P.items_sg1.end(),
                         [&](const WorkItem& x, const WorkItem& y) { return P.sq[x.q].nkb1 > P.sq[y.q].nkb1; });
        std::stable_sort(P.items_sg2.begin(), P.items_sg2.end(),
                         [&](const WorkItem& x, const WorkItem& y) { return P.sq[x.q].nkb2 > P.sq[y.q].nkb2; });
    }
    // byte layout from the chunk base
    size_t o = 0;
    auto region = [&](size_t& off, size_t bytes) {
        off = o;
        o = align256(o + bytes);
    };
    region(P.off_pairs, sizeof(DPair) * P.pairs.size());
    region(P.off_quartets, sizeof(DQuartet) * P.quartets.size());
    region(P.off_h, sizeof(WorkItem) * P.items_h.size());
    region(P.off_br, sizeof(WorkItem) * P.items_br.size());
    region(P.off_g1, sizeof(WorkItem) * P.items_g1.size());
    region(P.off_g2, sizeof(WorkItem) * P.items_g2.size());
    region(P.off_counters, sizeof(int) * 2 * GEMM_NVARIANT);
    region(P.off_srd, sizeof(SplitRowsDesc) * P.srd.size());
    region(P.off_sq, sizeof(SplitQuartet) * P.sq.size());
    region(P.off_sg1, sizeof(SplitGemmDesc) * P.sq.size());
    region(P.off_sg2, sizeof(SplitGemmDesc) * P.sq.size());
    region(P.off_isr, sizeof(WorkItem) * P.items_sr.size());
    region(P.off_isB, sizeof(WorkItem) * P.items_sB.size());
    region(P.off_isg1, sizeof(WorkItem) * P.items_sg1.size());
    region(P.off_isD, sizeof(WorkItem) * P.items_sD.size());
    region(P.off_isg2, sizeof(WorkItem) * P.items_sg2.size());
    P.off_data = o;
    // data regions: FP64 blocks in doubles from the workspace base, digit planes in bytes
    int64_t dw = (int64_t)((chunk_base + o) / 8);
    auto take = [&](int64_t ndoubles) {
        const int64_t at = dw;
        dw += ndoubles;
        dw = (dw + 31) & ~int64_t(31);
        return at;
    };
    for (auto& p : P.pairs) p.info_off = take(4 * (int64_t)p.Kab);
    for (auto& p : P.pairs) p.h_off = take((int64_t)p.nrow * p.Kab * p.np);
    for (auto& d : P.quartets) {
        d.rr_off = take((int64_t)d.kbra * d.kket * d.nr);
        d.x_off = take((int64_t)d.nab * d.kket * d.nq);
        if (jk && split) d.out_off = take((int64_t)d.nab * d.ncd);  // doubles from the workspace base
    }
    if (split) {
        auto take_bytes = [&](int64_t bytes) { return 8 * take((bytes + 7) / 8); };
        const int npair = (int)P.pairs.size();
        for (int p = 0; p < npair; ++p) {
            const DPair& pr = P.pairs[p];
            const int k = pr.Kab * pr.np, tb = split_tb(pr.nrow);
            SplitRowsDesc& r = P.srd[p];
            r.src_off = pr.h_off;
            r.dig_off = take_bytes(split_dig_bytes(pr.nrow, k, tb));
            r.exp_off = take_bytes(4 * (int64_t)split_rowpad(pr.nrow, tb));
            r.shift_off = take_bytes(4 * (int64_t)k);
            P.pairs[p].cs_off = r.shift_off;  // written by the pair's H kernel
        }
        for (size_t i = 0; i < P.quartets.size(); ++i) {
            const DQuartet& d = P.quartets[i];
            SplitQuartet& q = P.sq[i];
            const int k1 = d.kbra * d.np, k2 = d.kket * d.nq;
            const SplitRowsDesc &hb = P.srd[d.pb], &hk = P.srd[d.pk];
            q.a1_dig = take_bytes(split_dig_bytes(k2, k1, SPLIT_TA));
            q.a1_exp = take_bytes(4 * (int64_t)split_rowpad(k2, SPLIT_TA));
            q.b1_dig = hb.dig_off;
            q.b1_exp = hb.exp_off;
            q.a2_dig = take_bytes(split_dig_bytes(d.nab, k2, SPLIT_TA));
            q.a2_exp = take_bytes(4 * (int64_t)split_rowpad(d.nab, SPLIT_TA) * split_nseg(q.nkb2));
            q.b2_dig = hk.dig_off;
            q.b2_exp = hk.exp_off;
            q.c1_off = hb.shift_off;
            q.c2_off = hk.shift_off;
            SplitRowsDesc& rx = P.srd[npair + i];
            rx.src_off = d.x_off;
            rx.dig_off = q.a2_dig;
            rx.exp_off = q.a2_exp;
            rx.shift_off = q.c2_off;
            SplitGemmDesc g1{};
            g1.a_dig = q.a1_dig;
            g1.a_exp = q.a1_exp;
            g1.b_dig = q.b1_dig;
            g1.b_exp = q.b1_exp;
            g1.c_off = d.x_off;
            g1.M = k2;
            g1.N = d.nab;
            g1.nkb = q.nkb1;
            g1.ldc = k2;
            g1.transpose = 1;
            g1.tb = split_tb(d.nab);
            g1.a_nseg = 1;
            g1.nd = nd;
            P.sg1.push_back(g1);
            SplitGemmDesc g2{};
            g2.a_dig = q.a2_dig;
            g2.a_exp = q.a2_exp;
            g2.b_dig = q.b2_dig;
            g2.b_exp = q.b2_exp;
            g2.c_off = d.out_off;
            g2.M = d.nab;
            g2.N = d.ncd;
            g2.nkb = q.nkb2;
            g2.ldc = d.ncd;
            g2.transpose = 0;
            g2.tb = split_tb(d.ncd);
            g2.a_nseg = split_nseg(q.nkb2);  // X: one exponent per row and segment
            g2.nd = nd;
            P.sg2.push_back(g2);
        }
    }
    P.total = (size_t)dw * 8 - chunk_base;
    P.blob.assign(P.off_data, 0);
    auto put = [&](size_t off, const void* src, size_t bytes) {
        if (bytes) std::memcpy(P.blob.data() + off, src, bytes);
    };
    put(P.off_pairs, P.pairs.data(), sizeof(DPair) * P.pairs.size());
    put(P.off_quartets, P.quartets.data(), sizeof(DQuartet) * P.quartets.size());
    put(P.off_h, P.items_h.data(), sizeof(WorkItem) * P.items_h.size());
    put(P.off_br, P.items_br.data(), sizeof(WorkItem) * P.items_br.size());
    put(P.off_g1, P.items_g1.data(), sizeof(WorkItem) * P.items_g1.size());
    put(P.off_g2, P.items_g2.data(), sizeof(WorkItem) * P.items_g2.size());
    put(P.off_srd, P.srd.data(), sizeof(SplitRowsDesc) * P.srd.size());
    put(P.off_sq, P.sq.data(), sizeof(SplitQuartet) * P.sq.size());
    put(P.off_sg1, P.sg1.data(), sizeof(SplitGemmDesc) * P.sg1.size());
    put(P.off_sg2, P.sg2.data(), sizeof(SplitGemmDesc) * P.sg2.size());
    put(P.off_isr, P.items_sr.data(), sizeof(WorkItem) * P.items_sr.size());
    put(P.off_isB, P.items_sB.data(), sizeof(WorkItem) * P.items_sB.size());
    put(P.off_isg1, P.items_sg1.data(), sizeof(WorkItem) * P.items_sg1.size());
    put(P.off_isD, P.items_sD.data(), sizeof(WorkItem) * P.items_sD.size());
    put(P.off_isg2, P.items_sg2.data(), sizeof(WorkItem) * P.items_sg2.size());
}

// Workspace bytes that plan_chunks needs to keep quartets [b, e) in one chunk (an upper
// bound of the exact layout built by build_chunk).
size_t chunk_estimate(const lx_shell* sh, const lx_quartet* qs, int64_t b, int64_t e, int flags) {
    std::unordered_map<PairKey, int, PairKeyHash> seen;
    size_t used = CHUNK_SLACK;
    for (int64_t i = b; i < e; ++i) {
        const lx_quartet& q = qs[i];
        used += quartet_bytes(sh, q, flags);
        const PairKey kb{((int64_t)q.s[0] << 32 | (uint32_t)q.s[1]) * 2};
        const PairKey kk{((int64_t)q.s[2] << 32 | (uint32_t)q.s[3]) * 2 + 1};
        if (!seen.count(kb)) used += pair_bytes(sh, q.s[0], q.s[1], flags);
        if (!seen.count(kk)) used += pair_bytes(sh, q.s[2], q.s[3], flags);
        seen[kb] = 1;
        seen[kk] = 1;
    }
    return used;
}

int64_t prim_count(const lx_shell* sh, int32_t nshell) {
    int64_t n = 0;
    for (int32_t s = 0; s < nshell; ++s) n = std::max<int64_t>(n, (int64_t)sh[s].prim_offset + sh[s].nprim);
    return n;
}

// ------------------------------------------------------------------ plan + enqueue

// Host-side plan of one lx_eri_batch call: the head (shells, exponents, coefficients) and
// every chunk's descriptors, laid out for a workspace of `workspace_bytes`.
struct PlannedBatch {
    int flags = 0, nshell = 0, nprim = 0;
    size_t head = 0, o_exps = 0, o_coefs = 0, o_ncoef = 0;
    std::vector<char> head_blob;  // bytes [0, o_ncoef) of the workspace
    std::vector<ChunkPlan> chunks;
};

int plan_batch(const lx_shell* shells, int32_t nshell, const double* exps, const double* coefs, int32_t nprim_total,
               const lx_quartet* quartets, int64_t nquartet, int32_t flags, size_t workspace_bytes,
               const Overrides& ov, PlannedBatch& B) {
    B.flags = flags;
    B.nshell = nshell;
    B.nprim = nprim_total;
    B.head = head_bytes(nshell, nprim_total);
    if (workspace_bytes < B.head + CHUNK_SLACK) return LX_ERR_WORKSPACE;
    const int pflags = flags & (LX_SOLID | LX_PATH_SPLIT | JK_DIGEST | LX_SPLIT_DIGITS_MASK);
    std::vector<Chunk> chunks;
    int v = plan_chunks(shells, quartets, nquartet, pflags, workspace_bytes - B.head, chunks);
    if (v != LX_OK) return v;
    B.head_blob.assign(B.head, 0);
    DShell* dsh = reinterpret_cast<DShell*>(B.head_blob.data());
    int bf = 0;
    for (int32_t s = 0; s < nshell; ++s) {
        dsh[s].l = shells[s].l;
        dsh[s].K = shells[s].nprim;
        dsh[s].prim_off = shells[s].prim_offset;
        dsh[s].bf = bf;
        bf += nfun(shells[s].l, flags & LX_SOLID);
        for (int k = 0; k < 3; ++k) dsh[s].A[k] = shells[s].center[k];
    }
    B.o_exps = align256(sizeof(DShell) * (size_t)nshell);
    B.o_coefs = B.o_exps + align256(sizeof(double) * (size_t)nprim_total);
    B.o_ncoef = B.o_coefs + align256(sizeof(double) * (size_t)nprim_total);
    if (nprim_total > 0) {
        std::memcpy(B.head_blob.data() + B.o_exps, exps, sizeof(double) * (size_t)nprim_total);
        std::memcpy(B.head_blob.data() + B.o_coefs, coefs, sizeof(double) * (size_t)nprim_total);
    }
    B.chunks.resize(chunks.size());
    for (size_t c = 0; c < chunks.size(); ++c) {
        build_chunk(shells, quartets, chunks[c], pflags, B.head, B.chunks[c], ov);
        if (B.head + B.chunks[c].total > workspace_bytes) return LX_ERR_WORKSPACE;
    }
    return LX_OK;
}

// Density and outputs of lx_eri_jk (device pointers; J or K may be null).
struct JkArgs {
    const double* D;
    double* J;
    double* K;
    int64_t nbf;
};

// NVTX range over a scope (host side: marks when the work is enqueued; no-op without a tool)
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
};

// Enqueue a planned batch on stream st: the head upload, normalisation, then per chunk the
// descriptor upload and the kernels of the chosen path.  head_src / blob_src are the host
// bytes to upload (pageable, or pinned for graph capture).
int enqueue_batch(const PlannedBatch& B, const char* head_src, const std::vector<const char*>& blob_src, double* out,
                  void* workspace, unsigned* status, cudaStream_t st, bool time_stages, const JkArgs* jk) {
    const bool split = B.flags & LX_PATH_SPLIT, solid = B.flags & LX_SOLID;
    if ((B.flags & JK_DIGEST) && !jk) return LX_ERR_NULL;
    const NvtxRange range(split ? (jk ? "lx_eri split path, J/K" : "lx_eri split path")
                                : (jk ? "lx_eri FP64 path, J/K" : "lx_eri FP64 path"));
    if (jk) out = static_cast<double*>(workspace);  // blocks at workspace offsets, digested below
    const int nshell = B.nshell;
    char* wsb = static_cast<char*>(workspace);
    double* ws = static_cast<double*>(workspace);
    cudaError_t e = cudaMemcpyAsync(wsb, head_src, B.o_ncoef, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return cuda_fail(e);
    const DShell* d_sh = reinterpret_cast<const DShell*>(wsb);
    const double* d_exps = reinterpret_cast<const double*>(wsb + B.o_exps);
    const double* d_coefs = reinterpret_cast<const double*>(wsb + B.o_coefs);
    double* d_ncoef = reinterpret_cast<double*>(wsb + B.o_ncoef);
    StageTimer tm{time_stages, st};
    if ((e = tm.begin()) != cudaSuccess) return cuda_fail(e);
    if ((e = launch_norm(d_sh, nshell, d_exps, d_coefs, d_ncoef, status, st)) != cudaSuccess) return cuda_fail(e);
    if ((e = tm.end(LX_STAGE_NORM, 1)) != cudaSuccess) return cuda_fail(e);
    for (size_t c = 0; c < B.chunks.size(); ++c) {
        const NvtxRange chunk_range("lx_eri chunk");
        const ChunkPlan& P = B.chunks[c];
        char* base = wsb + B.head;
        e = cudaMemcpyAsync(base, blob_src[c], P.off_data, cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) return cuda_fail(e);
        const DPair* d_pairs = reinterpret_cast<const DPair*>(base + P.off_pairs);
        const DQuartet* d_q = reinterpret_cast<const DQuartet*>(base + P.off_quartets);
        const WorkItem* d_ih = reinterpret_cast<const WorkItem*>(base + P.off_h);
        const WorkItem* d_ibr = reinterpret_cast<const WorkItem*>(base + P.off_br);
        const WorkItem* d_ig1 = reinterpret_cast<const WorkItem*>(base + P.off_g1);
        const WorkItem* d_ig2 = reinterpret_cast<const WorkItem*>(base + P.off_g2);
        if ((e = tm.begin()) != cudaSuccess) return cuda_fail(e);
        if ((e = launch_pair_h(d_pairs, d_ih, (int)P.items_h.size(), d_sh, d_exps, d_ncoef, ws, ws, solid, split,
                               P.fold_lcap, P.fold_qcap, P.fold_wcap, P.fold_gcap, status, st)) != cudaSuccess)
            return cuda_fail(e);
        if ((e = tm.end(LX_STAGE_PAIR, 1)) != cudaSuccess) return cuda_fail(e);
        if ((e = tm.begin()) != cudaSuccess) return cuda_fail(e);
        if ((e = launch_boys_r(d_q, d_pairs, d_ibr, (int)P.items_br.size(), P.br_lmax, ws, status, st)) !=
            cudaSuccess)
            return cuda_fail(e);
        if ((e = tm.end(LX_STAGE_BOYS_R, 1)) != cudaSuccess) return cuda_fail(e);
        if (split) {
            auto at = [&](size_t off) { return base + off; };
            const SplitRowsDesc* d_srd = reinterpret_cast<const SplitRowsDesc*>(at(P.off_srd));
            const SplitQuartet* d_sq = reinterpret_cast<const SplitQuartet*>(at(P.off_sq));
            const SplitGemmDesc* d_sg1 = reinterpret_cast<const SplitGemmDesc*>(at(P.off_sg1));
            const SplitGemmDesc* d_sg2 = reinterpret_cast<const SplitGemmDesc*>(at(P.off_sg2));
            auto items = [&](size_t off) { return reinterpret_cast<const WorkItem*>(at(off)); };
            // operands of GEMM1 and the H operand of GEMM2: digit planes of [p|q]^T and of each
            // pair's H (H's column scales were written by the pair kernels)
            if ((e = tm.begin()) != cudaSuccess) return cuda_fail(e);
            if ((e = launch_split_operands(d_q, d_sq, items(P.off_isr), (int)P.items_sr.size(), d_srd,
                                           items(P.off_isB), (int)P.items_sB.size(), ws, wsb, st)) != cudaSuccess)
                return cuda_fail(e);
            if ((e = tm.end(LX_STAGE_SPLIT, 1)) != cudaSuccess) return cuda_fail(e);
            if ((e = tm.begin()) != cudaSuccess) return cuda_fail(e);
            if ((e = launch_split_gemm(d_sg1, items(P.off_isg1), (int)P.items_sg1.size(), wsb, ws, status, st,
                                       false, P.digits)) != cudaSuccess)
                return cuda_fail(e);
            if ((e = tm.end(LX_STAGE_GEMM1, 1)) != cudaSuccess) return cuda_fail(e);
            // the other operand of GEMM2: digit planes of [ab|q], one exponent per row and segment
            if ((e = tm.begin()) != cudaSuccess) return cuda_fail(e);
            if ((e = launch_split_rows(d_srd, items(P.off_isD), (int)P.items_sD.size(), ws, wsb, st)) != cudaSuccess)
                return cuda_fail(e);
            if ((e = tm.end(LX_STAGE_SPLIT, 1)) != cudaSuccess) return cuda_fail(e);
            if ((e = tm.begin()) != cudaSuccess) return cuda_fail(e);
            if ((e = launch_split_gemm(d_sg2, items(P.off_isg2), (int)P.items_sg2.size(), wsb, out, status, st,
                                       true, P.digits)) != cudaSuccess)
                return cuda_fail(e);
            if ((e = tm.end(LX_STAGE_GEMM2, 1)) != cudaSuccess) return cuda_fail(e);
        } else {
            if ((e = tm.begin()) != cudaSuccess) return cuda_fail(e);
            int* d_counters = reinterpret_cast<int*>(base + P.off_counters);
            if ((e = launch_gemm1(d_q, d_pairs, d_ig1, P.g1_counts, ws, d_counters, status, st)) != cudaSuccess)
                return cuda_fail(e);
            if ((e = tm.end(LX_STAGE_GEMM1, 1)) != cudaSuccess) return cuda_fail(e);
            if (jk) {
                // J and K straight from [ab|q]: no second transform, no stored block
                if ((e = tm.begin()) != cudaSuccess) return cuda_fail(e);
                if ((e = launch_jk_direct(d_q, d_pairs, d_sh, (int)P.quartets.size(), P.jkd_qc, P.jkd_smem, ws,
                                          solid, jk->D, jk->nbf, jk->J, jk->K, st)) != cudaSuccess)
                    return cuda_fail(e);
                if ((e = tm.end(LX_STAGE_DIGEST, 1)) != cudaSuccess) return cuda_fail(e);
                continue;
            }
            if ((e = tm.begin()) != cudaSuccess) return cuda_fail(e);
            if ((e = launch_gemm2(d_q, d_pairs, d_ig2, P.g2_counts, ws, out, d_counters + GEMM_NVARIANT, status,
                                  st)) != cudaSuccess)
                return cuda_fail(e);
            if ((e = tm.end(LX_STAGE_GEMM2, 1)) != cudaSuccess) return cuda_fail(e);
        }
        if (jk) {
            if ((e = tm.begin()) != cudaSuccess) return cuda_fail(e);
            if ((e = launch_jk_digest(d_q, d_pairs, d_sh, (int)P.quartets.size(), ws, solid, jk->D, jk->nbf, jk->J,
                                      jk->K, st)) != cudaSuccess)
                return cuda_fail(e);
            if ((e = tm.end(LX_STAGE_DIGEST, 1)) != cudaSuccess) return cuda_fail(e);
        }
    }
    return LX_OK;
}

}  // namespace
}  // namespace lx

using namespace lx;

namespace {

// Pinned staging buffers for the descriptor uploads of lx_eri_batch, per device: copies from
// pageable memory would make every call wait for the stream, so the planned descriptors are
// copied into a page-locked buffer first.  A buffer is held by one call from stage_acquire to
// stage_release, then read by that call's uploads until the event recorded after them has
// completed.  Up to STAGE_POOL buffers are kept per device; when none is free the least
// recently used one is waited for (more are made only if every buffer is held).
constexpr int STAGE_POOL = 4;
struct StageBuf {
    char* ptr = nullptr;
    size_t cap = 0;
    cudaEvent_t done = nullptr;
    uint64_t stamp = 0;    // order of last use
    bool held = false;     // between stage_acquire and stage_release
    bool pending = false;  // uploads enqueued, event not yet seen complete
};
std::mutex g_stage_mutex;
std::vector<StageBuf> g_stage[MAX_DEVICES];
uint64_t g_stage_clock = 0;

// Hold a pinned buffer of at least `bytes` that no enqueued copy still reads.
int stage_acquire(int dev, size_t bytes, int& idx, char*& ptr) {
    std::lock_guard<std::mutex> lock(g_stage_mutex);
    auto& pool = g_stage[dev];
    int best = -1, lru = -1;
    for (int i = 0; i < (int)pool.size(); ++i) {
        StageBuf& b = pool[i];
        if (b.held) continue;
        if (b.pending) {
            const cudaError_t q = cudaEventQuery(b.done);
            if (q == cudaSuccess) b.pending = false;
            else if (q != cudaErrorNotReady) return cuda_fail(q);
        }
        if (lru < 0 || b.stamp < pool[lru].stamp) lru = i;
        if (!b.pending && b.cap >= bytes && (best < 0 || b.cap < pool[best].cap)) best = i;
    }
    if (best < 0) {
        if ((int)pool.size() < STAGE_POOL || lru < 0) {
            pool.emplace_back();
            best = (int)pool.size() - 1;
            cudaError_t e = cudaEventCreateWithFlags(&pool[best].done, cudaEventDisableTiming);
            if (e != cudaSuccess) {
                pool.pop_back();
                return cuda_fail(e);
            }
        } else {
            best = lru;
        }
        StageBuf& b = pool[best];
        if (b.pending) {
            cudaError_t e = cudaEventSynchronize(b.done);
            if (e != cudaSuccess) return cuda_fail(e);
            b.pending = false;
        }
        if (b.cap < bytes) {
            if (b.ptr) {
                cudaError_t e = cudaFreeHost(b.ptr);
                if (e != cudaSuccess) return cuda_fail(e);
                b.ptr = nullptr;
                b.cap = 0;
            }
            const size_t cap = std::max(bytes, (size_t)1 << 20);
            cudaError_t e = cudaHostAlloc(reinterpret_cast<void**>(&b.ptr), cap, cudaHostAllocDefault);
            if (e != cudaSuccess) return cuda_fail(e);
            b.cap = cap;
        }
    }
    StageBuf& b = pool[best];
    b.held = true;
    b.stamp = ++g_stage_clock;
    idx = best;
    ptr = b.ptr;
    return LX_OK;
}

// Give buffer idx back; its uploads (if any were enqueued) end at an event recorded on st.
int stage_release(int dev, int idx, cudaStream_t st, bool enqueued) {
    std::lock_guard<std::mutex> lock(g_stage_mutex);
    StageBuf& b = g_stage[dev][idx];
    b.held = false;
    if (!enqueued) return LX_OK;
    cudaError_t e = cudaEventRecord(b.done, st);
    if (e != cudaSuccess) {
        // the uploads may still be in flight: wait for the stream before the buffer is reused
        cudaStreamSynchronize(st);
        return cuda_fail(e);
    }
    b.pending = true;
    return LX_OK;
}

}  // namespace

namespace lx {

const FoldHost* fold_tables() { return g_fold_ready ? &g_fold : nullptr; }

int report_cuda_error(cudaError_t e) { return cuda_fail(e); }

int entry_prepare(void* cuda_stream, const char* who, unsigned** status) {
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    const cudaError_t e = cudaStreamIsCapturing(static_cast<cudaStream_t>(cuda_stream), &cap);
    if (e != cudaSuccess) return cuda_fail(e);
    if (cap != cudaStreamCaptureStatusNone) {
        std::snprintf(t_cuda_msg, sizeof(t_cuda_msg), "%s on a capturing stream: its uploads read host memory "
                      "released when the call returns", who);
        return LX_ERR_CUDA;
    }
    return ensure_device(status);
}

// lx_eri_batch without the pinned staging: the descriptors are uploaded straight from the
// planner's host vectors (the copies then wait for the stream).  Allocates nothing.
int eri_batch_unstaged(const lx_shell* shells, int32_t nshell, const double* exps, const double* coefs,
                       int32_t nprim_total, const lx_quartet* quartets, int64_t nquartet, int32_t flags, double* out,
                       void* workspace, size_t workspace_bytes, void* cuda_stream) {
    int v = validate(shells, nshell, exps, coefs, nprim_total, quartets, nquartet, flags, true);
    if (v != LX_OK) return v;
    if (nquartet == 0) return LX_OK;
    if (!out) return LX_ERR_NULL;
    if (!workspace || (reinterpret_cast<uintptr_t>(workspace) & 255)) return LX_ERR_WORKSPACE;
    unsigned* status = nullptr;
    if ((v = ensure_device(&status)) != LX_OK) return v;
    PlannedBatch B;
    if ((v = plan_batch(shells, nshell, exps, coefs, nprim_total, quartets, nquartet, flags, workspace_bytes,
                        Overrides(), B)) != LX_OK)
        return v;
    std::vector<const char*> blobs;
    for (const auto& P : B.chunks) blobs.push_back(P.blob.data());
    return enqueue_batch(B, B.head_blob.data(), blobs, out, workspace, status, static_cast<cudaStream_t>(cuda_stream),
                         (flags & LX_TIME_STAGES) != 0, nullptr);
}

}  // namespace lx

namespace {

// Routing network of LX_PATH_ROUTED per device (FP16 parameters on the device, thresholds of
// the 4-, 5- and 6-digit split tiers on the predicted log10 split error).
std::mutex g_router_mutex;
void* g_router_params[MAX_DEVICES];
float g_router_tau[MAX_DEVICES][LX_ROUTE_NTIER];

// Workspace the routed call needs before the batches run: features and predictions.
size_t routed_scratch_bytes(int64_t n) {
    return align256(sizeof(float) * LX_MLP_NIN * (size_t)n) + align256(sizeof(float) * LX_MLP_NOUT * (size_t)n);
}

// Plan one batch, stage its descriptors in pinned memory and enqueue it (inputs validated,
// device set up, stream not capturing).
int eri_batch_staged(const lx_shell* shells, int32_t nshell, const double* exps, const double* coefs,
                     int32_t nprim_total, const lx_quartet* quartets, int64_t nquartet, int32_t flags, double* out,
                     void* workspace, size_t workspace_bytes, cudaStream_t st, unsigned* status,
                     const JkArgs* jk = nullptr) {
    PlannedBatch B;
    int v = plan_batch(shells, nshell, exps, coefs, nprim_total, quartets, nquartet, flags, workspace_bytes,
                       Overrides(), B);
    if (v != LX_OK) return v;
    // descriptors into a pinned staging buffer, so that the uploads do not wait for the stream
    size_t total = align256(B.head_blob.size());
    for (const auto& P : B.chunks) total += align256(P.blob.size());
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e);
    int idx = -1;
    char* stage = nullptr;
    if ((v = stage_acquire(dev, total, idx, stage)) != LX_OK) return v;
    std::memcpy(stage, B.head_blob.data(), B.head_blob.size());
    const char* head_src = stage;
    size_t o = align256(B.head_blob.size());
    std::vector<const char*> blobs;
    for (const auto& P : B.chunks) {
        std::memcpy(stage + o, P.blob.data(), P.blob.size());
        blobs.push_back(stage + o);
        o += align256(P.blob.size());
    }
    v = enqueue_batch(B, head_src, blobs, out, workspace, status, st, (flags & LX_TIME_STAGES) != 0, jk);
    const int r = stage_release(dev, idx, st, true);
    return v != LX_OK ? v : r;
}

// The quartet list of the bra-list x ket-list form: quartet i nket + j = (bra pair i | ket
// pair j), output block i nket + j of a dense [nbra][nket][n_ab][n_cd] array.  Checks the
// shells (without primitives), the pair indices and that each list has one class.
int expand_pairs(const lx_shell* shells, int32_t nshell, const int32_t* bra, int64_t nbra, const int32_t* ket,
                 int64_t nket, int32_t flags, std::vector<lx_quartet>& qs) {
    qs.clear();
    int v = validate(shells, nshell, nullptr, nullptr, 0, nullptr, 0, flags, false);
    if (v != LX_OK) return v;
    if (nbra < 0 || nket < 0) return LX_ERR_SIZE;
    if (nbra == 0 || nket == 0) return LX_OK;
    if (!bra || !ket) return LX_ERR_NULL;
    if (nbra > LX_PAIRS_MAX_QUARTETS / nket) return LX_ERR_SIZE;
    auto check = [&](const int32_t* pr, int64_t n) {
        for (int64_t i = 0; i < 2 * n; ++i)
            if (pr[i] < 0 || pr[i] >= nshell) return LX_ERR_QUARTET;
        for (int64_t i = 1; i < n; ++i)
            if (shells[pr[2 * i]].l != shells[pr[0]].l || shells[pr[2 * i + 1]].l != shells[pr[1]].l)
                return LX_ERR_PAIR_CLASS;
        return LX_OK;
    };
    if ((v = check(bra, nbra)) != LX_OK || (v = check(ket, nket)) != LX_OK) return v;
    const bool solid = flags & LX_SOLID;
    const int64_t block = (int64_t)nfun(shells[bra[0]].l, solid) * nfun(shells[bra[1]].l, solid) *
                          nfun(shells[ket[0]].l, solid) * nfun(shells[ket[1]].l, solid);
    qs.resize((size_t)(nbra * nket));
    for (int64_t i = 0; i < nbra; ++i)
        for (int64_t j = 0; j < nket; ++j) {
            lx_quartet& q = qs[(size_t)(i * nket + j)];
            q.s[0] = bra[2 * i];
            q.s[1] = bra[2 * i + 1];
            q.s[2] = ket[2 * j];
            q.s[3] = ket[2 * j + 1];
            q.out_offset = (i * nket + j) * block;
        }
    return LX_OK;
}

// lx_eri_workspace_size (least = false) and lx_eri_workspace_min (least = true); extra is 0
// or JK_DIGEST (not a caller flag: added after validation).
int64_t workspace_need(const lx_shell* shells, int32_t nshell, const lx_quartet* quartets, int64_t nquartet,
                       int32_t flags, int32_t extra, bool least) {
    const int v = validate(shells, nshell, nullptr, nullptr, 0, quartets, nquartet, flags, false);
    if (v != LX_OK) return v;
    const size_t head = head_bytes(nshell, (int32_t)prim_count(shells, nshell));
    const int32_t solid = (flags & LX_SOLID) | extra;
    // a routed quartet may take either path; the predictions come first
    const bool routed = flags & LX_PATH_ROUTED;
    auto est = [&](int64_t b, int64_t e) {
        if (routed)
            return std::max(chunk_estimate(shells, quartets, b, e, solid),
                            chunk_estimate(shells, quartets, b, e, solid | LX_PATH_SPLIT));
        return chunk_estimate(shells, quartets, b, e, solid | (flags & LX_PATH_SPLIT));
    };
    size_t need = CHUNK_SLACK;
    if (!least)
        need = est(0, nquartet);
    else
        for (int64_t i = 0; i < nquartet; ++i) need = std::max(need, est(i, i + 1));
    const size_t total = head + need;
    return (int64_t)(routed ? std::max(total, routed_scratch_bytes(nquartet)) : total);
}

// lx_eri_batch, and lx_eri_jk with jk set (flags then carry JK_DIGEST and out is unused).
int eri_entry(const lx_shell* shells, int32_t nshell, const double* exps, const double* coefs, int32_t nprim_total,
              const lx_quartet* quartets, int64_t nquartet, int32_t flags, double* out, void* workspace,
              size_t workspace_bytes, void* cuda_stream, const JkArgs* jk) {
    const int32_t internal = flags & JK_DIGEST;
    flags &= ~JK_DIGEST;
    int v = validate(shells, nshell, exps, coefs, nprim_total, quartets, nquartet, flags, true);
    if (v != LX_OK) return v;
    flags |= internal;
    if (nquartet == 0) return LX_OK;
    if (!out && !jk) return LX_ERR_NULL;
    if (!workspace || (reinterpret_cast<uintptr_t>(workspace) & 255)) return LX_ERR_WORKSPACE;
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    cudaError_t e = cudaStreamIsCapturing(st, &cap);
    if (e != cudaSuccess) return cuda_fail(e);
    if (cap != cudaStreamCaptureStatusNone) {
        // the staging buffers are reused by later calls, so a captured upload would replay stale
        // descriptors: capture goes through lx_eri_graph_create, which owns its copies
        std::snprintf(t_cuda_msg, sizeof(t_cuda_msg), "lx_eri_batch on a capturing stream: use lx_eri_graph_create");
        return LX_ERR_CUDA;
    }
    unsigned* status = nullptr;
    if ((v = ensure_device(&status)) != LX_OK) return v;
    if (!(flags & LX_PATH_ROUTED))
        return eri_batch_staged(shells, nshell, exps, coefs, nprim_total, quartets, nquartet, flags, out, workspace,
                                workspace_bytes, st, status, jk);
    // routed: predictions into the (still unused) workspace, read back, then one staged batch
    // per path over the same output and workspace
    int dev = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return cuda_fail(e);
    const void* params = nullptr;
    float tau[LX_ROUTE_NTIER];
    {
        std::lock_guard<std::mutex> lock(g_router_mutex);
        params = g_router_params[dev];
        for (int t = 0; t < LX_ROUTE_NTIER; ++t) tau[t] = g_router_tau[dev][t];
    }
    if (!params) return LX_ERR_NO_ROUTER;
    if (workspace_bytes < routed_scratch_bytes(nquartet)) return LX_ERR_WORKSPACE;
    float* feat = static_cast<float*>(workspace);
    float* pred = reinterpret_cast<float*>(static_cast<char*>(workspace) +
                                           align256(sizeof(float) * LX_MLP_NIN * (size_t)nquartet));
    if ((v = lx_route_features(shells, nshell, exps, nprim_total, quartets, nquartet, feat, cuda_stream)) != LX_OK)
        return v;
    if ((e = launch_mlp_forward(params, feat, nquartet, pred, st)) != cudaSuccess) return cuda_fail(e);
    std::vector<float> hp((size_t)LX_MLP_NOUT * nquartet);
    if ((e = cudaMemcpyAsync(hp.data(), pred, sizeof(float) * LX_MLP_NOUT * nquartet, cudaMemcpyDeviceToHost, st)) !=
        cudaSuccess)
        return cuda_fail(e);
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return cuda_fail(e);
    // sub-batches: FP64, then the split tiers of 4, 5 and 6 digits
    std::vector<lx_quartet> sub[1 + LX_ROUTE_NTIER];
    const bool solid = flags & LX_SOLID;
    for (int64_t i = 0; i < nquartet; ++i) {
        const lx_quartet& q = quartets[i];
        const lx_shell &a = shells[q.s[0]], &b = shells[q.s[1]], &c = shells[q.s[2]], &d = shells[q.s[3]];
        const double nab = (double)nfun(a.l, solid) * nfun(b.l, solid), ncd = (double)nfun(c.l, solid) * nfun(d.l, solid);
        const double kp = (double)a.nprim * b.nprim * pyr(a.l + b.l), kq = (double)c.nprim * d.nprim * pyr(c.l + d.l);
        const double flop = 2.0 * nab * kp * kq + 2.0 * nab * kq * ncd;
        const float err = hp[(size_t)LX_MLP_NOUT * i + 1];  // predicted log10 split error (6 digits)
        int dst = 0;
        if (flop >= LX_ROUTE_SPLIT_MIN_FLOP)
            for (int t = 0; t < LX_ROUTE_NTIER; ++t)
                if (err < tau[t]) {
                    dst = 1 + t;
                    break;
                }
        sub[dst].push_back(q);
    }
    const int32_t base = flags & ~LX_PATH_ROUTED;
    for (int k = 0; k <= LX_ROUTE_NTIER; ++k) {
        if (sub[k].empty()) continue;
        const int32_t f = k == 0 ? base : base | LX_PATH_SPLIT | LX_SPLIT_DIGITS(SPLIT_MIN_DIGITS + k - 1);
        if ((v = eri_batch_staged(shells, nshell, exps, coefs, nprim_total, sub[k].data(), (int64_t)sub[k].size(), f,
                                  out, workspace, workspace_bytes, st, status, jk)) != LX_OK)
            return v;
    }
    return LX_OK;
}

}  // namespace

extern "C" {

int64_t lx_eri_out_size(const lx_shell* shells, int32_t nshell, const lx_quartet* quartets, int64_t nquartet,
                        int32_t flags) {
    const int v = validate(shells, nshell, nullptr, nullptr, 0, quartets, nquartet, flags, false);
    if (v != LX_OK) return v;
    const bool solid = flags & LX_SOLID;
    int64_t n = 0;
    for (int64_t i = 0; i < nquartet; ++i) {
        int64_t sz = 1;
        for (int k = 0; k < 4; ++k) sz *= nfun(shells[quartets[i].s[k]].l, solid);
        n = std::max(n, quartets[i].out_offset + sz);
    }
    return n;
}

int64_t lx_eri_workspace_size(const lx_shell* shells, int32_t nshell, const lx_quartet* quartets, int64_t nquartet,
                              int32_t flags) {
    return workspace_need(shells, nshell, quartets, nquartet, flags, 0, false);
}

int64_t lx_eri_workspace_min(const lx_shell* shells, int32_t nshell, const lx_quartet* quartets, int64_t nquartet,
                             int32_t flags) {
    return workspace_need(shells, nshell, quartets, nquartet, flags, 0, true);
}

int lx_eri_batch(const lx_shell* shells, int32_t nshell, const double* exps, const double* coefs,
                 int32_t nprim_total, const lx_quartet* quartets, int64_t nquartet, int32_t flags, double* out,
                 void* workspace, size_t workspace_bytes, void* cuda_stream) {
    if (flags & JK_DIGEST) return LX_ERR_FLAGS;
    return eri_entry(shells, nshell, exps, coefs, nprim_total, quartets, nquartet, flags, out, workspace,
                     workspace_bytes, cuda_stream, nullptr);
}

int lx_router_set(const void* params_f16, const float* tau) {
    if (!params_f16 || !tau) return LX_ERR_NULL;
    for (int t = 0; t < LX_ROUTE_NTIER; ++t)
        if (!std::isfinite(tau[t])) return LX_ERR_SIZE;
    unsigned* status = nullptr;
    int v = ensure_device(&status);
    if (v != LX_OK) return v;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e);
    std::lock_guard<std::mutex> lock(g_router_mutex);
    if (!g_router_params[dev]) {
        void* p = nullptr;
        if ((e = cudaMalloc(&p, 2 * (size_t)LX_MLP_NPARAM)) != cudaSuccess) return cuda_fail(e);
        g_router_params[dev] = p;
    }
    // synchronous: no batch on any stream may read the parameters while they are replaced
    if ((e = cudaDeviceSynchronize()) != cudaSuccess) return cuda_fail(e);
    if ((e = cudaMemcpy(g_router_params[dev], params_f16, 2 * (size_t)LX_MLP_NPARAM, cudaMemcpyHostToDevice)) !=
        cudaSuccess)
        return cuda_fail(e);
    for (int t = 0; t < LX_ROUTE_NTIER; ++t) g_router_tau[dev][t] = tau[t];
    return LX_OK;
}

namespace {
struct GraphHandle {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    std::vector<void*> pinned;
    int device = 0;
};

// Device milliseconds per stage of the LX_TIME_STAGES work on stream st (clears it).
int collect_stage_ms(cudaStream_t st, double* ms) {
    for (int i = 0; i < LX_NSTAGE; ++i) ms[i] = 0.0;
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e);
    std::lock_guard<std::mutex> lock(g_timing_mutex);
    std::vector<PendingTiming> keep;
    for (const auto& p : g_pending) {
        if (p.stream != st) {
            keep.push_back(p);
            continue;
        }
        float t = 0.f;
        if (cudaEventElapsedTime(&t, p.begin, p.end) == cudaSuccess) ms[p.stage] += t;
        cudaEventDestroy(p.begin);
        cudaEventDestroy(p.end);
    }
    g_pending.swap(keep);
    return LX_OK;
}
}  // namespace

int lx_eri_graph_create(const lx_shell* shells, int32_t nshell, const double* exps, const double* coefs,
                        int32_t nprim_total, const lx_quartet* quartets, int64_t nquartet, int32_t flags,
                        double* out, void* workspace, size_t workspace_bytes, void** handle) {
    if (!handle) return LX_ERR_NULL;
    *handle = nullptr;
    if (flags & (LX_TIME_STAGES | LX_PATH_ROUTED)) return LX_ERR_FLAGS;
    int v = validate(shells, nshell, exps, coefs, nprim_total, quartets, nquartet, flags, true);
    if (v != LX_OK) return v;
    if (!out) return LX_ERR_NULL;
    if (!workspace || (reinterpret_cast<uintptr_t>(workspace) & 255)) return LX_ERR_WORKSPACE;
    unsigned* status = nullptr;
    if ((v = ensure_device(&status)) != LX_OK) return v;
    PlannedBatch B;
    if ((v = plan_batch(shells, nshell, exps, coefs, nprim_total, quartets, nquartet, flags, workspace_bytes,
                        Overrides(), B)) != LX_OK)
        return v;
    GraphHandle* h = new GraphHandle();
    cudaGetDevice(&h->device);
    auto fail = [&](int code) {
        for (void* p : h->pinned) cudaFreeHost(p);
        if (h->exec) cudaGraphExecDestroy(h->exec);
        if (h->graph) cudaGraphDestroy(h->graph);
        delete h;
        return code;
    };
    // host bytes the graph's copy nodes read: pinned and owned by the handle
    auto pin = [&](const std::vector<char>& src, const char** dst) {
        void* p = nullptr;
        cudaError_t e = cudaHostAlloc(&p, src.size() > 0 ? src.size() : 1, cudaHostAllocDefault);
        if (e != cudaSuccess) return e;
        if (!src.empty()) std::memcpy(p, src.data(), src.size());
        h->pinned.push_back(p);
        *dst = static_cast<const char*>(p);
        return cudaSuccess;
    };
    const char* head_src = nullptr;
    std::vector<const char*> blobs(B.chunks.size());
    cudaError_t e = pin(B.head_blob, &head_src);
    for (size_t c = 0; e == cudaSuccess && c < B.chunks.size(); ++c) e = pin(B.chunks[c].blob, &blobs[c]);
    if (e != cudaSuccess) return fail(cuda_fail(e));
    cudaStream_t cs = nullptr;
    if ((e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking)) != cudaSuccess) return fail(cuda_fail(e));
    if ((e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal)) != cudaSuccess) {
        cudaStreamDestroy(cs);
        return fail(cuda_fail(e));
    }
    v = nquartet > 0 ? enqueue_batch(B, head_src, blobs, out, workspace, status, cs, false, nullptr) : LX_OK;
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(cs, &g);
    cudaStreamDestroy(cs);
    h->graph = g;
    if (v != LX_OK) return fail(v);
    if (e != cudaSuccess) return fail(cuda_fail(e));
    if ((e = cudaGraphInstantiate(&h->exec, h->graph, 0)) != cudaSuccess) return fail(cuda_fail(e));
    *handle = h;
    return LX_OK;
}

int lx_eri_graph_launch(void* handle, void* cuda_stream) {
    if (!handle) return LX_ERR_NULL;
    GraphHandle* h = static_cast<GraphHandle*>(handle);
    cudaError_t e = cudaGraphLaunch(h->exec, static_cast<cudaStream_t>(cuda_stream));
    return e == cudaSuccess ? LX_OK : cuda_fail(e);
}

int lx_eri_graph_destroy(void* handle) {
    if (!handle) return LX_OK;
    GraphHandle* h = static_cast<GraphHandle*>(handle);
    for (void* p : h->pinned) cudaFreeHost(p);
    if (h->exec) cudaGraphExecDestroy(h->exec);
    if (h->graph) cudaGraphDestroy(h->graph);
    delete h;
    return LX_OK;
}

int lx_eri_autotune(const lx_shell* shells, int32_t nshell, const double* exps, const double* coefs,
                    int32_t nprim_total, const lx_quartet* quartets, int64_t nquartet, int32_t flags, double* out,
                    int64_t out_doubles, void* workspace, size_t workspace_bytes, int32_t max_keys, int32_t samples,
                    void* cuda_stream) {
    int v = validate(shells, nshell, exps, coefs, nprim_total, quartets, nquartet, flags, true);
    if (v != LX_OK) return v;
    if (flags & LX_PATH_ROUTED) return LX_ERR_FLAGS;
    if (flags & LX_PATH_SPLIT) return LX_OK;  // the split path has one tile shape
    if (max_keys < 1 || samples < 1 || out_doubles < 0) return LX_ERR_SIZE;
    if (!out || !workspace) return LX_ERR_NULL;
    unsigned* status = nullptr;
    if ((v = ensure_device(&status)) != LX_OK) return v;
    const bool solid = flags & LX_SOLID;
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    // group by key; the costliest keys (total GEMM1 work) first
    std::map<TuneKey, std::vector<int64_t>> groups;
    std::map<TuneKey, double> cost;
    for (int64_t i = 0; i < nquartet; ++i) {
        const TuneKey k = tune_key(shells, quartets[i], solid);
        groups[k].push_back(i);
        cost[k] += (double)nfun(k.la, solid) * nfun(k.lb, solid) * k.kbra * pyr(k.la + k.lb) * k.kket * pyr(k.lc + k.ld);
    }
    std::vector<std::pair<double, TuneKey>> order;
    for (const auto& kv : cost) order.push_back({-kv.second, kv.first});
    std::sort(order.begin(), order.end(), [](const auto& x, const auto& y) { return x.first < y.first; });
    int tuned = 0;
    for (const auto& ok : order) {
        if (tuned >= max_keys) break;
        const std::vector<int64_t>& idx = groups[ok.second];
        std::vector<lx_quartet> sub;
        int64_t pos = 0;
        for (size_t j = 0; j < idx.size() && (int)j < samples; ++j) {
            lx_quartet q = quartets[idx[j]];
            int64_t sz = 1;
            for (int k = 0; k < 4; ++k) sz *= nfun(shells[q.s[k]].l, solid);
            if (pos + sz > out_doubles) break;
            q.out_offset = pos;
            pos += sz;
            sub.push_back(q);
        }
        if (sub.empty()) continue;
        double best1 = 1e300, best2 = 1e300;
        int v1 = GEMM_V32x64, v2 = GEMM_V32x64;
        for (int var = 0; var < GEMM_NVARIANT; ++var) {
            PlannedBatch B;
            Overrides ov;
            ov.v1 = ov.v2 = var;
            if ((v = plan_batch(shells, nshell, exps, coefs, nprim_total, sub.data(), (int64_t)sub.size(),
                                flags & (LX_SOLID | LX_PATH_SPLIT), workspace_bytes, ov, B)) != LX_OK)
                return v;
            std::vector<const char*> blobs;
            for (const auto& P : B.chunks) blobs.push_back(P.blob.data());
            double t1 = 1e300, t2 = 1e300;
            for (int rep = 0; rep < 3; ++rep) {  // first repetition warms up
                if ((v = enqueue_batch(B, B.head_blob.data(), blobs, out, workspace, status, st, true, nullptr)) !=
                    LX_OK)
                    return v;
                double ms[LX_NSTAGE];
                if ((v = collect_stage_ms(st, ms)) != LX_OK) return v;
                if (rep > 0) {
                    t1 = std::min(t1, ms[LX_STAGE_GEMM1]);
                    t2 = std::min(t2, ms[LX_STAGE_GEMM2]);
                }
            }
            if (t1 < best1) {
                best1 = t1;
                v1 = var;
            }
            if (t2 < best2) {
                best2 = t2;
                v2 = var;
            }
        }
        std::lock_guard<std::mutex> lock(g_tune_mutex);
        g_tune[ok.second] = TuneVal{v1, v2};
        ++tuned;
    }
    return LX_OK;
}

int64_t lx_tune_export(int32_t* rows, int64_t cap) {
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    int64_t n = 0;
    for (const auto& kv : g_tune) {
        if (rows && n < cap) {
            const TuneKey& k = kv.first;
            int32_t* r = rows + 9 * n;
            r[0] = k.la, r[1] = k.lb, r[2] = k.lc, r[3] = k.ld, r[4] = k.kbra, r[5] = k.kket, r[6] = k.solid;
            r[7] = kv.second.v1, r[8] = kv.second.v2;
        }
        ++n;
    }
    return n;
}

int lx_tune_import(const int32_t* rows, int64_t n) {
    if (n < 0) return LX_ERR_SIZE;
    if (n > 0 && !rows) return LX_ERR_NULL;
    for (int64_t i = 0; i < n; ++i) {
        const int32_t* r = rows + 9 * i;
        for (int k = 0; k < 4; ++k)
            if (r[k] < 0 || r[k] > LX_LMAX) return LX_ERR_SIZE;
        if (r[4] < 1 || r[5] < 1 || r[6] < 0 || r[6] > 1 || r[7] < 0 || r[7] >= GEMM_NVARIANT || r[8] < 0 ||
            r[8] >= GEMM_NVARIANT)
            return LX_ERR_SIZE;
    }
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    for (int64_t i = 0; i < n; ++i) {
        const int32_t* r = rows + 9 * i;
        g_tune[TuneKey{r[0], r[1], r[2], r[3], r[4], r[5], r[6]}] = TuneVal{r[7], r[8]};
    }
    return LX_OK;
}

int lx_tune_clear(void) {
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    g_tune.clear();
    return LX_OK;
}

int lx_eri_sync_status(void* cuda_stream) {
    unsigned* status = nullptr;
    int v = ensure_device(&status);
    if (v != LX_OK) return v;
    cudaError_t e = cudaStreamSynchronize(static_cast<cudaStream_t>(cuda_stream));
    if (e != cudaSuccess) return cuda_fail(e);
    unsigned word = 0;
    if ((e = cudaMemcpyFromSymbol(&word, g_status_word, sizeof(word))) != cudaSuccess) return cuda_fail(e);
    if (word) {
        const unsigned zero = 0;
        if ((e = cudaMemcpyToSymbol(g_status_word, &zero, sizeof(zero))) != cudaSuccess) return cuda_fail(e);
        return LX_ERR_DEVICE_STATUS;
    }
    return LX_OK;
}

int lx_eri_stage_times(double* ms, int64_t* launches, int32_t nstage, void* cuda_stream) {
    if (nstage < 0 || nstage > LX_NSTAGE) return LX_ERR_SIZE;
    if (nstage > 0 && !ms) return LX_ERR_NULL;
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e);
    for (int i = 0; i < nstage; ++i) {
        ms[i] = 0.0;
        if (launches) launches[i] = 0;
    }
    std::lock_guard<std::mutex> lock(g_timing_mutex);
    std::vector<PendingTiming> keep;
    int rc = LX_OK;
    for (const auto& p : g_pending) {
        if (p.stream != st) {
            keep.push_back(p);
            continue;
        }
        float t = 0.f;
        e = cudaEventElapsedTime(&t, p.begin, p.end);
        if (e != cudaSuccess) rc = cuda_fail(e);
        if (p.stage < nstage) {
            ms[p.stage] += t;
            if (launches) launches[p.stage] += p.launches;
        }
        cudaEventDestroy(p.begin);
        cudaEventDestroy(p.end);
    }
    g_pending.swap(keep);
    return rc;
}

int64_t lx_eri_pairs_out_size(const lx_shell* shells, int32_t nshell, const int32_t* bra_pairs, int64_t nbra,
                              const int32_t* ket_pairs, int64_t nket, int32_t flags) {
    std::vector<lx_quartet> qs;
    const int v = expand_pairs(shells, nshell, bra_pairs, nbra, ket_pairs, nket, flags, qs);
    if (v != LX_OK) return v;
    return qs.empty() ? 0 : lx_eri_out_size(shells, nshell, qs.data(), (int64_t)qs.size(), flags);
}

int64_t lx_eri_pairs_workspace_size(const lx_shell* shells, int32_t nshell, const int32_t* bra_pairs, int64_t nbra,
                                    const int32_t* ket_pairs, int64_t nket, int32_t flags) {
    std::vector<lx_quartet> qs;
    const int v = expand_pairs(shells, nshell, bra_pairs, nbra, ket_pairs, nket, flags, qs);
    if (v != LX_OK) return v;
    return lx_eri_workspace_size(shells, nshell, qs.data(), (int64_t)qs.size(), flags);
}

int64_t lx_eri_pairs_workspace_min(const lx_shell* shells, int32_t nshell, const int32_t* bra_pairs, int64_t nbra,
                                   const int32_t* ket_pairs, int64_t nket, int32_t flags) {
    std::vector<lx_quartet> qs;
    const int v = expand_pairs(shells, nshell, bra_pairs, nbra, ket_pairs, nket, flags, qs);
    if (v != LX_OK) return v;
    return lx_eri_workspace_min(shells, nshell, qs.data(), (int64_t)qs.size(), flags);
}

int lx_eri_pairs(const lx_shell* shells, int32_t nshell, const double* exps, const double* coefs, int32_t nprim_total,
                 const int32_t* bra_pairs, int64_t nbra, const int32_t* ket_pairs, int64_t nket, int32_t flags,
                 double* out, void* workspace, size_t workspace_bytes, void* cuda_stream) {
    std::vector<lx_quartet> qs;
    const int v = expand_pairs(shells, nshell, bra_pairs, nbra, ket_pairs, nket, flags, qs);
    if (v != LX_OK) return v;
    return lx_eri_batch(shells, nshell, exps, coefs, nprim_total, qs.data(), (int64_t)qs.size(), flags, out,
                        workspace, workspace_bytes, cuda_stream);
}

int64_t lx_nbf(const lx_shell* shells, int32_t nshell, int32_t flags) {
    const int v = validate(shells, nshell, nullptr, nullptr, 0, nullptr, 0, flags, false);
    if (v != LX_OK) return v;
    int64_t n = 0;
    for (int32_t s = 0; s < nshell; ++s) n += nfun(shells[s].l, flags & LX_SOLID);
    return n;
}

int64_t lx_eri_jk_workspace_size(const lx_shell* shells, int32_t nshell, const lx_quartet* quartets,
                                 int64_t nquartet, int32_t flags) {
    return workspace_need(shells, nshell, quartets, nquartet, flags, JK_DIGEST, false);
}

int64_t lx_eri_jk_workspace_min(const lx_shell* shells, int32_t nshell, const lx_quartet* quartets,
                                int64_t nquartet, int32_t flags) {
    return workspace_need(shells, nshell, quartets, nquartet, flags, JK_DIGEST, true);
}

int lx_eri_jk(const lx_shell* shells, int32_t nshell, const double* exps, const double* coefs, int32_t nprim_total,
              const lx_quartet* quartets, int64_t nquartet, int32_t flags, const double* D, double* J, double* K,
              void* workspace, size_t workspace_bytes, void* cuda_stream) {
    const int64_t nbf = lx_nbf(shells, nshell, flags);
    if (nbf < 0) return (int)nbf;
    if (nbf > INT32_MAX) return LX_ERR_SIZE;
    if (nquartet > 0 && (!D || (!J && !K))) return LX_ERR_NULL;
    const JkArgs jk{D, J, K, nbf};
    return eri_entry(shells, nshell, exps, coefs, nprim_total, quartets, nquartet, flags | JK_DIGEST, nullptr,
                     workspace, workspace_bytes, cuda_stream, &jk);
}

int lx_selftest_timeout(uint64_t tries, void* cuda_stream) {
    if (tries > (1ull << 24)) return LX_ERR_SIZE;
    unsigned* status = nullptr;
    const int v = ensure_device(&status);
    if (v != LX_OK) return v;
    const cudaError_t e = launch_wait_selftest(status, tries, static_cast<cudaStream_t>(cuda_stream));
    return e == cudaSuccess ? LX_OK : cuda_fail(e);
}

const char* lx_strerror(int code) {
    switch (code) {
        case LX_OK: return "success";
        case LX_ERR_NULL: return "a required pointer is NULL";
        case LX_ERR_SHELL: return "invalid shell (l, nprim, reserved field, primitive range or center)";
        case LX_ERR_PRIMITIVE: return "invalid primitive (exponent must be finite and > 0, coefficient finite)";
        case LX_ERR_QUARTET: return "invalid quartet (shell index out of range or negative out_offset)";
        case LX_ERR_FLAGS: return "unknown flag bits";
        case LX_ERR_WORKSPACE: return "workspace NULL, misaligned or too small";
        case LX_ERR_CUDA: return "CUDA runtime error";
        case LX_ERR_ARCH: return "current device is not compute capability 10.3 (GB300)";
        case LX_ERR_DEVICE_STATUS: return "a kernel reported a bad index or input";
        case LX_ERR_SIZE: return "a size argument is negative or too large";
        case LX_ERR_STATIC_SCRATCH: return "batch needs more scratch than the static array of lx_eri_batch_static holds";
        case LX_ERR_NO_ROUTER: return "LX_PATH_ROUTED without a routing network (lx_router_set)";
        case LX_ERR_PAIR_CLASS: return "a pair list mixes angular momenta (every bra pair, and every ket pair, needs the same (l, l'))";
        default: return "unknown error code";
    }
}

const char* lx_last_cuda_error(void) { return t_cuda_msg; }

int lx_boys(int32_t mmax, const double* T, int64_t n, double* F, void* cuda_stream) {
    if (mmax < 0 || mmax > LTOT || n < 0) return LX_ERR_SIZE;
    if (n > 0 && (!T || !F)) return LX_ERR_NULL;
    unsigned* status = nullptr;
    int v = ensure_device(&status);
    if (v != LX_OK) return v;
    cudaError_t e = launch_boys(mmax, T, n, F, status, static_cast<cudaStream_t>(cuda_stream));
    return e == cudaSuccess ? LX_OK : cuda_fail(e);
}

int lx_hermite_R(int32_t L, const double* params, int64_t n, double* R, void* cuda_stream) {
    if (L < 0 || L > LTOT || n < 0) return LX_ERR_SIZE;
    if (n > 0 && (!params || !R)) return LX_ERR_NULL;
    unsigned* status = nullptr;
    int v = ensure_device(&status);
    if (v != LX_OK) return v;
    cudaError_t e = launch_hermite_r(L, params, n, R, status, static_cast<cudaStream_t>(cuda_stream));
    return e == cudaSuccess ? LX_OK : cuda_fail(e);
}

int lx_hermite_H(const lx_shell* shells, int32_t nshell, const double* exps, const double* coefs,
                 int32_t nprim_total, const int32_t* pairs, int32_t npair, int32_t flags, double* H, int64_t stride,
                 void* cuda_stream) {
    const int32_t side = (flags & 0x100) ? 1 : 0;
    const int32_t f = flags & ~0x100;
    int v = validate(shells, nshell, exps, coefs, nprim_total, nullptr, 0, f, true);
    if (v != LX_OK) return v;
    if (npair < 0 || stride < 0) return LX_ERR_SIZE;
    if (npair == 0) return LX_OK;
    if (!pairs || !H) return LX_ERR_NULL;
    const bool solid = f & LX_SOLID;
    int64_t need = 0;
    for (int32_t k = 0; k < npair; ++k) {
        const int sa = pairs[2 * k], sb = pairs[2 * k + 1];
        if (sa < 0 || sa >= nshell || sb < 0 || sb >= nshell) return LX_ERR_QUARTET;
        need = std::max<int64_t>(need, (int64_t)nfun(shells[sa].l, solid) * nfun(shells[sb].l, solid) *
                                           shells[sa].nprim * shells[sb].nprim * pyr(shells[sa].l + shells[sb].l));
    }
    if (stride < need) return LX_ERR_SIZE;
    unsigned* status = nullptr;
    if ((v = ensure_device(&status)) != LX_OK) return v;
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    // Scratch for descriptors and pair scalars, stream-ordered.
    std::vector<DPair> dp(npair);
    std::vector<WorkItem> items;
    int64_t info_total = 0;
    for (int32_t k = 0; k < npair; ++k) {
        const int sa = pairs[2 * k], sb = pairs[2 * k + 1];
        DPair& p = dp[k];
        p.sa = sa;
        p.sb = sb;
        p.Kab = shells[sa].nprim * shells[sb].nprim;
        p.nrow = nfun(shells[sa].l, solid) * nfun(shells[sb].l, solid);
        p.np = pyr(shells[sa].l + shells[sb].l);
        p.sign = side;
        p.solid = solid ? 1 : 0;
        p.cs_off = -1;
        p.info_off = info_total;
        info_total += 4 * (int64_t)p.Kab;
        for (int kp = 0; kp < p.Kab; ++kp) items.push_back({k, kp, 0, 0});
    }
    const size_t o_sh = 0, o_exps = align256(sizeof(DShell) * (size_t)nshell);
    const size_t o_coefs = o_exps + align256(8 * (size_t)nprim_total);
    const size_t o_ncoef = o_coefs + align256(8 * (size_t)nprim_total);
    const size_t o_pairs = o_ncoef + align256(8 * (size_t)nprim_total);
    const size_t o_items = o_pairs + align256(sizeof(DPair) * (size_t)npair);
    const size_t o_info = o_items + align256(sizeof(WorkItem) * items.size());
    const size_t scratch_bytes = o_info + align256(8 * (size_t)info_total);
    char* scratch = nullptr;
    cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(&scratch), scratch_bytes, st);
    if (e != cudaSuccess) return cuda_fail(e);
    for (int32_t k = 0; k < npair; ++k) dp[k].h_off = (int64_t)k * stride;
    std::vector<char> blob(o_info, 0);
    DShell* dsh = reinterpret_cast<DShell*>(blob.data() + o_sh);
    for (int32_t s = 0; s < nshell; ++s) {
        dsh[s].l = shells[s].l;
        dsh[s].K = shells[s].nprim;
        dsh[s].prim_off = shells[s].prim_offset;
        for (int k = 0; k < 3; ++k) dsh[s].A[k] = shells[s].center[k];
    }
    std::memcpy(blob.data() + o_exps, exps, 8 * (size_t)nprim_total);
    std::memcpy(blob.data() + o_coefs, coefs, 8 * (size_t)nprim_total);
    std::memcpy(blob.data() + o_pairs, dp.data(), sizeof(DPair) * dp.size());
    std::memcpy(blob.data() + o_items, items.data(), sizeof(WorkItem) * items.size());
    if ((e = cudaMemcpyAsync(scratch, blob.data(), o_info, cudaMemcpyHostToDevice, st)) != cudaSuccess)
        return cuda_fail(e);
    const DShell* d_sh = reinterpret_cast<const DShell*>(scratch + o_sh);
    const double* d_exps = reinterpret_cast<const double*>(scratch + o_exps);
    const double* d_coefs = reinterpret_cast<const double*>(scratch + o_coefs);
    double* d_ncoef = reinterpret_cast<double*>(scratch + o_ncoef);
    if ((e = launch_norm(d_sh, nshell, d_exps, d_coefs, d_ncoef, status, st)) != cudaSuccess) return cuda_fail(e);
    int lcap = 0, qcap = 0, wcap = 0, gcap = 0;
    if (solid)
        for (const DPair& pr : dp) {
            const FoldPairTab& t = g_fold.pair[shells[pr.sa].l][shells[pr.sb].l];
            lcap = std::max(lcap, std::max(shells[pr.sa].l, shells[pr.sb].l));
            qcap = std::max(qcap, t.maxq + 1);
            wcap = std::max(wcap, t.maxw);
            gcap = std::max(gcap, t.maxg + 1);
        }
    if ((e = launch_pair_h(reinterpret_cast<const DPair*>(scratch + o_pairs),
                           reinterpret_cast<const WorkItem*>(scratch + o_items), (int)items.size(), d_sh, d_exps,
                           d_ncoef, H, reinterpret_cast<double*>(scratch + o_info), solid, false, lcap, qcap, wcap, gcap, status,
                           st)) !=
        cudaSuccess)
        return cuda_fail(e);
    if ((e = cudaFreeAsync(scratch, st)) != cudaSuccess) return cuda_fail(e);
    return LX_OK;
}

int lx_split_gemm(int32_t M, int32_t N, int32_t K, const double* A, int32_t lda, const double* B, int32_t ldb,
                  double* C, int32_t ldc, int32_t digits, void* cuda_stream) {
    if (M < 1 || N < 1 || K < 1 || K > (1 << 20) || lda < K || ldb < K || ldc < N) return LX_ERR_SIZE;
    if (digits < SPLIT_MIN_DIGITS || digits > SPLIT_NSLICE) return LX_ERR_SIZE;
    if (!A || !B || !C) return LX_ERR_NULL;
    unsigned* status = nullptr;
    int v = ensure_device(&status);
    if (v != LX_OK) return v;
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    const int nkb = split_nkb(K);
    const int tb = split_tb(N);
    const int ra = split_rowpad(M, SPLIT_TA), rb = split_rowpad(N, tb);
    std::vector<SplitRowsDesc> rd(2);
    rd[0] = SplitRowsDesc{0, 0, 0, -1, lda, M, K, SPLIT_TA, nkb, 0, 0, 0, digits, 0};
    rd[1] = SplitRowsDesc{0, 0, 0, -1, ldb, N, K, tb, nkb, 0, 0, 0, digits, 0};
    std::vector<WorkItem> ia, ib, ig;
    for (int r = 0; r < ra; r += 8) ia.push_back({0, r, 0, 0});
    for (int r = 0; r < rb; r += 8) ib.push_back({1, r, 0, 0});
    for (int m = 0; m < ra / SPLIT_TA; ++m)
        for (int n = 0; n < (N + tb - 1) / tb; ++n) ig.push_back({0, m, n, 0});
    size_t o = 0;
    auto region = [&](size_t bytes) {
        const size_t at = o;
        o = align256(o + bytes);
        return at;
    };
    const size_t o_rd = region(sizeof(SplitRowsDesc) * 2), o_g = region(sizeof(SplitGemmDesc));
    const size_t o_ia = region(sizeof(WorkItem) * ia.size()), o_ib = region(sizeof(WorkItem) * ib.size());
    const size_t o_ig = region(sizeof(WorkItem) * ig.size());
    const size_t blob_bytes = o;
    rd[0].dig_off = (int64_t)region((size_t)split_dig_bytes(M, K, SPLIT_TA));
    rd[0].exp_off = (int64_t)region(4 * (size_t)ra);
    rd[1].dig_off = (int64_t)region((size_t)split_dig_bytes(N, K, tb));
    rd[1].exp_off = (int64_t)region(4 * (size_t)rb);
    SplitGemmDesc g{};
    g.a_dig = rd[0].dig_off;
    g.a_exp = rd[0].exp_off;
    g.b_dig = rd[1].dig_off;
    g.b_exp = rd[1].exp_off;
    g.M = M;
    g.N = N;
    g.nkb = nkb;
    g.ldc = ldc;
    g.tb = tb;
    g.a_nseg = 1;
    g.nd = digits;
    std::vector<char> blob(blob_bytes, 0);
    std::memcpy(blob.data() + o_rd, rd.data(), sizeof(SplitRowsDesc) * 2);
    std::memcpy(blob.data() + o_g, &g, sizeof(g));
    std::memcpy(blob.data() + o_ia, ia.data(), sizeof(WorkItem) * ia.size());
    std::memcpy(blob.data() + o_ib, ib.data(), sizeof(WorkItem) * ib.size());
    std::memcpy(blob.data() + o_ig, ig.data(), sizeof(WorkItem) * ig.size());
    char* scratch = nullptr;
    cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(&scratch), o, st);
    if (e != cudaSuccess) return cuda_fail(e);
    if ((e = cudaMemcpyAsync(scratch, blob.data(), blob_bytes, cudaMemcpyHostToDevice, st)) != cudaSuccess)
        return cuda_fail(e);
    const SplitRowsDesc* d_rd = reinterpret_cast<const SplitRowsDesc*>(scratch + o_rd);
    if ((e = launch_split_rows(d_rd, reinterpret_cast<const WorkItem*>(scratch + o_ia), (int)ia.size(), A, scratch,
                               st)) != cudaSuccess)
        return cuda_fail(e);
    if ((e = launch_split_rows(d_rd, reinterpret_cast<const WorkItem*>(scratch + o_ib), (int)ib.size(), B, scratch,
                               st)) != cudaSuccess)
        return cuda_fail(e);
    if ((e = launch_split_gemm(reinterpret_cast<const SplitGemmDesc*>(scratch + o_g),
                               reinterpret_cast<const WorkItem*>(scratch + o_ig), (int)ig.size(), scratch, C, status,
                               st, false, digits)) != cudaSuccess)
        return cuda_fail(e);
    if ((e = cudaFreeAsync(scratch, st)) != cudaSuccess) return cuda_fail(e);
    return LX_OK;
}

int lx_route_features(const lx_shell* shells, int32_t nshell, const double* exps, int32_t nprim_total,
                      const lx_quartet* quartets, int64_t nquartet, float* feat, void* cuda_stream) {
    // coefficients are not used: pass the exponents twice to reuse the validation
    int v = validate(shells, nshell, exps, exps, nprim_total, quartets, nquartet, 0, true);
    if (v != LX_OK) return v;
    if (nquartet == 0) return LX_OK;
    if (!feat) return LX_ERR_NULL;
    unsigned* status = nullptr;
    if ((v = ensure_device(&status)) != LX_OK) return v;
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    const size_t o_sh = 0, o_ex = align256(sizeof(DShell) * (size_t)nshell);
    const size_t o_q = o_ex + align256(8 * (size_t)nprim_total), total = o_q + align256(16 * (size_t)nquartet);
    std::vector<char> blob(total, 0);
    DShell* dsh = reinterpret_cast<DShell*>(blob.data() + o_sh);
    for (int32_t s = 0; s < nshell; ++s) {
        dsh[s].l = shells[s].l;
        dsh[s].K = shells[s].nprim;
        dsh[s].prim_off = shells[s].prim_offset;
        for (int k = 0; k < 3; ++k) dsh[s].A[k] = shells[s].center[k];
    }
    std::memcpy(blob.data() + o_ex, exps, 8 * (size_t)nprim_total);
    int* q4 = reinterpret_cast<int*>(blob.data() + o_q);
    for (int64_t i = 0; i < nquartet; ++i)
        for (int k = 0; k < 4; ++k) q4[4 * i + k] = quartets[i].s[k];
    char* scratch = nullptr;
    cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(&scratch), total, st);
    if (e != cudaSuccess) return cuda_fail(e);
    if ((e = cudaMemcpyAsync(scratch, blob.data(), total, cudaMemcpyHostToDevice, st)) != cudaSuccess)
        return cuda_fail(e);
    if ((e = launch_features(reinterpret_cast<const DShell*>(scratch + o_sh),
                             reinterpret_cast<const double*>(scratch + o_ex), reinterpret_cast<const int*>(scratch + o_q),
                             nquartet, feat, st)) != cudaSuccess)
        return cuda_fail(e);
    if ((e = cudaFreeAsync(scratch, st)) != cudaSuccess) return cuda_fail(e);
    return LX_OK;
}

int lx_mlp_forward(const void* params_f16, const float* feat, int64_t n, float* out, void* cuda_stream) {
    if (n < 0) return LX_ERR_SIZE;
    if (n > 0 && (!params_f16 || !feat || !out)) return LX_ERR_NULL;
    unsigned* status = nullptr;
    int v = ensure_device(&status);
    if (v != LX_OK) return v;
    cudaError_t e = launch_mlp_forward(params_f16, feat, n, out, static_cast<cudaStream_t>(cuda_stream));
    return e == cudaSuccess ? LX_OK : cuda_fail(e);
}

int lx_mlp_grad(const float* params, const float* feat, const float* target, int64_t n, float* grad, float* loss,
                void* cuda_stream) {
    if (n < 0) return LX_ERR_SIZE;
    if (!params || !grad || !loss || (n > 0 && (!feat || !target))) return LX_ERR_NULL;
    unsigned* status = nullptr;
    int v = ensure_device(&status);
    if (v != LX_OK) return v;
    cudaError_t e = launch_mlp_grad(params, feat, target, n, grad, loss, static_cast<cudaStream_t>(cuda_stream));
    return e == cudaSuccess ? LX_OK : cuda_fail(e);
}

int lx_mlp_adam(float* params, float* m, float* v, float* grad, void* params_f16, int32_t step, float lr, float beta1,
                float beta2, float eps, void* cuda_stream) {
    if (step < 1) return LX_ERR_SIZE;
    if (!params || !m || !v || !grad || !params_f16) return LX_ERR_NULL;
    unsigned* status = nullptr;
    int rc = ensure_device(&status);
    if (rc != LX_OK) return rc;
    cudaError_t e = launch_mlp_adam(params, m, v, grad, params_f16, step, lr, beta1, beta2, eps,
                                    static_cast<cudaStream_t>(cuda_stream));
    return e == cudaSuccess ? LX_OK : cuda_fail(e);
}

}  // extern "C"
