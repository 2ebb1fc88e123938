// Host-side generation of the library's constant tables.
//
// Real solid harmonics are built by the standard recurrences for regular solid
// harmonics (Helgaker, Jorgensen & Olsen, Molecular Electronic-Structure Theory,
// Eqs. 6.4.70-6.4.73), starting from S_00 = 1:
//   S_{l+1,l+1}  = sqrt(2^{d(l,0)} (2l+1)/(2l+2)) (x S_{l,l} - (1 - d(l,0)) y S_{l,-l})
//   S_{l+1,-l-1} = sqrt(2^{d(l,0)} (2l+1)/(2l+2)) (y S_{l,l} + (1 - d(l,0)) x S_{l,-l})
//   S_{l+1,m}    = ((2l+1) z S_{l,m} - sqrt((l+m)(l-m)) r^2 S_{l-1,m}) / sqrt((l+m+1)(l-m+1))
// and each is rescaled to a unit-normalised Gaussian on x^l-normalised Cartesians
// (the matrices C^a_{lm} of the paper's Section 2 that fold into H).
//
// The Boys table holds F_n(T_k) (Eq. boys) on a uniform grid for a Taylor expansion;
// values come from the series F_n(T) = exp(-T) sum_k (2T)^k / ((2n+1)(2n+3)...(2n+2k+1))
// for the top order, summed in long double, and the downward recursion
// F_n = (2T F_{n+1} + exp(-T)) / (2n+1).
#include <algorithm>
#include <array>
#include <cmath>
#include <map>
#include <tuple>
#include <vector>

#include "lx_internal.cuh"

namespace lx {

namespace {

using Mono = std::tuple<int, int, int>;
using Poly = std::map<Mono, long double>;

Poly mul_var(const Poly& p, int axis, long double s) {
    Poly r;
    for (const auto& [m, c] : p) {
        auto [a, b, d] = m;
        if (axis == 0) ++a;
        else if (axis == 1) ++b;
        else ++d;
        r[{a, b, d}] += s * c;
    }
    return r;
}

void add_to(Poly& acc, const Poly& p, long double s) {
    for (const auto& [m, c] : p) acc[m] += s * c;
}

long double dfact_odd(int n) {  // (2n-1)!!
    long double r = 1.0L;
    for (int k = 2 * n - 1; k > 1; k -= 2) r *= k;
    return r;
}

// S[l][m + l] for l = 0..LMAX as polynomials.
std::vector<std::vector<Poly>> solid_polys() {
    std::vector<std::vector<Poly>> S(LMAX + 1);
    S[0] = {Poly{{{0, 0, 0}, 1.0L}}};
    for (int l = 0; l < LMAX; ++l) {
        S[l + 1].assign(2 * l + 3, Poly{});
        const long double d0 = (l == 0) ? 1.0L : 0.0L;
        const long double f = std::sqrt(std::pow(2.0L, d0) * (2 * l + 1) / (2.0L * l + 2));
        Poly top = mul_var(S[l][2 * l], 0, f);                    // x S_{l,l}
        Poly bot = mul_var(S[l][2 * l], 1, f);                    // y S_{l,l}
        if (l > 0) {
            add_to(top, mul_var(S[l][0], 1, f), -1.0L);           // - y S_{l,-l}
            add_to(bot, mul_var(S[l][0], 0, f), 1.0L);            // + x S_{l,-l}
        }
        S[l + 1][2 * (l + 1)] = top;
        S[l + 1][0] = bot;
        for (int m = -l; m <= l; ++m) {
            Poly p = mul_var(S[l][m + l], 2, 2 * l + 1);          // (2l+1) z S_{l,m}
            if (l >= 1 && m >= -(l - 1) && m <= l - 1) {
                const long double g = std::sqrt((long double)(l + m) * (l - m));
                const Poly& q = S[l - 1][m + l - 1];
                for (int axis = 0; axis < 3; ++axis) add_to(p, mul_var(mul_var(q, axis, 1.0L), axis, 1.0L), -g);
            }
            const long double h = 1.0L / std::sqrt((long double)(l + m + 1) * (l - m + 1));
            Poly r;
            for (const auto& [mo, c] : p) r[mo] = c * h;
            S[l + 1][m + l + 1] = r;
        }
    }
    return S;
}

}  // namespace

int solid_offset(int l) {
    int off = 0;
    for (int k = 0; k < l; ++k) off += (2 * k + 1) * ncart(k);
    return off;
}

void make_solid_coefs(double* out) {
    auto S = solid_polys();
    for (int l = 0; l <= LMAX; ++l) {
        const int nc = ncart(l);
        std::vector<Mono> comps;
        for (int i = 0; i <= l; ++i)
            for (int j = 0; j <= i; ++j) comps.emplace_back(l - i, i - j, j);
        for (int m = -l; m <= l; ++m) {
            std::vector<long double> v(nc, 0.0L);
            for (const auto& [mo, c] : S[l][m + l]) {
                for (int k = 0; k < nc; ++k)
                    if (comps[k] == mo) v[k] += c;
            }
            // Gaussian self-overlap in units where <x^l|x^l> = (2l-1)!!:
            // <x^a y^b z^c | x^a' y^b' z^c'> is the product of (n-1)!! over the even sums n.
            long double nrm = 0.0L;
            for (int p = 0; p < nc; ++p)
                for (int q = 0; q < nc; ++q) {
                    auto [a0, a1, a2] = comps[p];
                    auto [b0, b1, b2] = comps[q];
                    if ((a0 + b0) & 1 || (a1 + b1) & 1 || (a2 + b2) & 1) continue;
                    nrm += v[p] * v[q] * dfact_odd((a0 + b0) / 2) * dfact_odd((a1 + b1) / 2) *
                           dfact_odd((a2 + b2) / 2);
                }
            const long double s = std::sqrt(dfact_odd(l) / nrm);
            for (int k = 0; k < nc; ++k) out[solid_offset(l) + (m + l) * nc + k] = (double)(v[k] * s);
        }
    }
}

void make_boys_table(double* table) {
    const int ntop = BOYS_NROW - 1;
    for (int k = 0; k < BOYS_NPT; ++k) {
        const long double T = k * (long double)BOYS_DT;
        const long double e = std::exp(-T);
        long double term = 1.0L / (2 * ntop + 1), sum = term;
        for (int i = 1; i < 100000; ++i) {
            term *= 2.0L * T / (2 * ntop + 2 * i + 1);
            sum += term;
            if (term < 1e-25L * sum && i > T) break;
        }
        long double f = e * sum;
        table[ntop * BOYS_NPT + k] = (double)f;
        for (int n = ntop - 1; n >= 0; --n) {
            f = (2.0L * T * f + e) / (2 * n + 1);
            table[n * BOYS_NPT + k] = (double)f;
        }
    }
}

namespace {

// Sort rows by decreasing length (stable), take them in groups of 32 and append one stream
// per warp (the layout described with FoldSeg) to ent, and the FOLD_NWARP + 1 stream bounds
// to wstart; returns the position of each original row.
std::vector<int> emit_groups(const std::vector<std::vector<int>>& rows, int null_entry, std::vector<int>& wstart,
                             std::vector<int>& ent) {
    const int n = (int)rows.size(), ngroup = (n + 31) / 32;
    std::vector<int> order(n), pos(n);
    for (int i = 0; i < n; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(),
                     [&](int a, int b) { return rows[a].size() > rows[b].size(); });
    for (int i = 0; i < n; ++i) pos[order[i]] = i;
    for (int w = 0; w < FOLD_NWARP; ++w) {
        wstart.push_back((int)ent.size());
        std::vector<std::array<int, 32>> cols;  // the warp's columns in stream order
        for (int k = 0, g; (g = fold_group(k, w)) < ngroup; ++k) {
            size_t len = 1;  // a group of empty rows still ends with one (null) column
            for (int i = 32 * g; i < std::min(n, 32 * g + 32); ++i) len = std::max(len, rows[order[i]].size());
            for (size_t j = 0; j < len; ++j) {
                std::array<int, 32> c;
                bool any = false;
                for (int i = 0; i < 32; ++i) {
                    const int r = 32 * g + i;
                    const bool real = r < n && j < rows[order[r]].size();
                    c[i] = real ? rows[order[r]][j] : null_entry;
                    any = any || real;
                }
                for (int i = 0; i < 32; ++i) c[i] |= (any ? 0 : FOLD_SKIP) | (j + 1 == len ? FOLD_FLAG : 0);
                cols.push_back(c);
            }
        }
        std::array<int, 32> pad;
        pad.fill(null_entry | FOLD_SKIP);
        while (cols.size() % 4) cols.push_back(pad);
        for (size_t q = 0; q < cols.size(); q += 4)
            for (int i = 0; i < 32; ++i)
                for (int k = 0; k < 4; ++k) ent.push_back(cols[q + k][i]);
    }
    wstart.push_back((int)ent.size());
    return pos;
}

}  // namespace

constexpr int W_PLACEHOLDER = FOLD_MASK;  // never a real W entry

bool make_fold_lists(const double* coefs, FoldHost& F) {
    F.wstart.clear();
    F.g_rec.clear();
    F.q_ent.clear();
    F.w_ent.clear();
    F.h_ent.clear();
    F.h_out.clear();
    F.segs.clear();
    bool ok = true;
    for (int la = 0; la <= LMAX; ++la)
        for (int lb = 0; lb <= LMAX; ++lb) {
            const int nca = ncart(la), ncb = ncart(lb), nsa = 2 * la + 1, nsb = 2 * lb + 1;
            const int nt = la + lb + 1, np = pyr(la + lb), sb1 = lb + 1;
            std::vector<int> ax(nca), ay(nca), az(nca), bidx((lb + 1) * (lb + 1), -1);
            for (int i = 0, k = 0; i <= la; ++i)
                for (int j = 0; j <= i; ++j, ++k) {
                    ax[k] = la - i;
                    ay[k] = i - j;
                    az[k] = j;
                }
            for (int i = 0, k = 0; i <= lb; ++i)
                for (int j = 0; j <= i; ++j, ++k) bidx[(lb - i) * (lb + 1) + (i - j)] = k;  // (bx, by) -> b
            std::vector<int> lsum(np);  // t + u + v of Hermite index p
            for (int L = 0; L <= la + lb; ++L)
                for (int p = L ? pyr(L - 1) : 0; p < pyr(L); ++p) lsum[p] = L;
            const double* Ca = coefs + solid_offset(la);
            const double* Cb = coefs + solid_offset(lb);
            // distinct (ay, az) of shell a, in component order
            std::vector<std::pair<int, int>> yz;
            for (int k = 0; k < nca; ++k)
                if (std::find(yz.begin(), yz.end(), std::make_pair(ay[k], az[k])) == yz.end())
                    yz.emplace_back(ay[k], az[k]);
            FoldPairTab& tab = F.pair[la][lb];
            tab.seg0 = (int)F.segs.size();
            tab.maxq = tab.maxw = tab.maxg = 0;
            const size_t w_first = F.w_ent.size();
            for (int mb = 0; mb < nsb; ++mb) {
                FoldSeg sg{};
                sg.h_row0 = (int)F.h_out.size();
                // Q rows, keyed (ay, az, bx, u, v); their G entries C_b[m_b][b] E^z_{az bz v},
                // numbered in order of first use
                std::vector<std::tuple<int, int, int, int, int>> qkey;
                std::vector<std::vector<int>> qrows;
                std::map<int, int> gidx_of;  // (coefficient index | E^z index << 10) -> G index
                std::vector<int> grec;
                for (const auto& [y, z] : yz)
                    for (int bx = 0; bx <= lb; ++bx)
                        for (int u = 0; u <= y + lb - bx; ++u)
                            for (int v = 0; v <= z + lb - bx; ++v) {
                                std::vector<int> row;
                                for (int by = 0; by <= lb - bx; ++by) {
                                    const int bz = lb - bx - by, b = bidx[bx * (lb + 1) + by];
                                    if (std::fabs(Cb[mb * ncb + b]) <= 1e-14 || u > y + by || v > z + bz) continue;
                                    const int rec = (mb * ncb + b) | (((z * sb1 + bz) * nt + v) << 10);
                                    auto gi = gidx_of.find(rec);
                                    if (gi == gidx_of.end()) {
                                        gi = gidx_of.emplace(rec, (int)grec.size()).first;
                                        grec.push_back(rec);
                                    }
                                    row.push_back(gi->second | (((y * sb1 + by) * nt + u) << 10));
                                }
                                if (row.empty()) continue;
                                qkey.emplace_back(y, z, bx, u, v);
                                qrows.push_back(std::move(row));
                            }
                sg.q_nrow = (int)qkey.size();
                if (sg.q_nrow > FOLD_QMAX) return false;
                sg.g_n = (int)grec.size();
                if (sg.g_n > FOLD_GMAX) return false;
                sg.g_off = (int)F.g_rec.size();
                F.g_rec.insert(F.g_rec.end(), grec.begin(), grec.end());
                // padding entries take the zero stored after the G entries (G index g_n)
                sg.q_ws = (int)F.wstart.size();
                const std::vector<int> qpos = emit_groups(qrows, sg.g_n, F.wstart, F.q_ent);
                // W rows, keyed (a, p)
                std::vector<std::vector<int>> wrows;
                std::vector<int> wrow((size_t)nca * np, -1);
                for (int a = 0; a < nca; ++a) {
                    std::vector<std::vector<int>> rows(np);
                    for (int qi = 0; qi < (int)qkey.size(); ++qi) {
                        const auto [y, z, bx, u, v] = qkey[qi];
                        if (y != ay[a] || z != az[a]) continue;
                        for (int t = 0; t <= ax[a] + bx; ++t)
                            rows[hidx(t, u, v)].push_back(((ax[a] * sb1 + bx) * nt + t) | (qpos[qi] << 10));
                    }
                    for (int p = 0; p < np; ++p) {
                        if (rows[p].empty()) continue;
                        wrow[(size_t)a * np + p] = (int)wrows.size();
                        wrows.push_back(std::move(rows[p]));
                    }
                }
                sg.w_nrow = (int)wrows.size();
                if (sg.w_nrow > FOLD_WMAX) return false;
                // padding entries point at the zero Q row, known once every m_b is built
                sg.w_ws = (int)F.wstart.size();
                const std::vector<int> wpos = emit_groups(wrows, W_PLACEHOLDER, F.wstart, F.w_ent);
                // H rows (m_a, p); the output position travels with the row
                std::vector<std::vector<int>> hrows;
                std::vector<int> hkey;
                for (int ma = 0; ma < nsa; ++ma)
                    for (int p = 0; p < np; ++p) {
                        std::vector<int> row;
                        for (int a = 0; a < nca; ++a) {
                            const int w = wrow[(size_t)a * np + p];
                            if (w < 0 || std::fabs(Ca[ma * nca + a]) <= 1e-14) continue;
                            row.push_back((ma * nca + a) | (wpos[w] << 10));
                        }
                        hrows.push_back(std::move(row));
                        hkey.push_back(ma | (p << 4) | ((lsum[p] & 1) << 30));
                    }
                // padding entries take the zero stored after C_a (coefficient index nsa nca)
                sg.h_ws = (int)F.wstart.size();
                const std::vector<int> hpos = emit_groups(hrows, nsa * nca, F.wstart, F.h_ent);
                std::vector<int> out(hrows.size());
                for (size_t i = 0; i < hrows.size(); ++i) out[hpos[i]] = hkey[i];
                F.h_out.insert(F.h_out.end(), out.begin(), out.end());
                tab.maxq = std::max(tab.maxq, sg.q_nrow);
                tab.maxg = std::max(tab.maxg, sg.g_n);
                tab.maxw = std::max(tab.maxw, sg.w_nrow);
                F.segs.push_back(sg);
            }
            for (size_t i = w_first; i < F.w_ent.size(); ++i)  // E^x[0] times the zero row, flags kept
                if ((F.w_ent[i] & FOLD_MASK) == W_PLACEHOLDER) F.w_ent[i] = (F.w_ent[i] & ~FOLD_MASK) | (tab.maxq << 10);
        }
    return ok;
}

void make_tuv_table(int* tuv) {
    for (int n = 0; n <= LTOT; ++n)
        for (int i = 0; i <= n; ++i)
            for (int v = 0; v <= i; ++v) {
                const int u = i - v, t = n - i;
                tuv[hidx(t, u, v)] = t | (u << 8) | (v << 16);
            }
}


}  // namespace lx
