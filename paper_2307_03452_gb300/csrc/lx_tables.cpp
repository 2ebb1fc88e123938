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

void make_solid_classes(const double* coefs, SolidClassTab* tab) {
    for (int l = 0; l <= LMAX; ++l) {
        SolidClassTab& T = tab[l];
        T = SolidClassTab{};
        const int nc = ncart(l);
        const double* C = coefs + solid_offset(l);
        int key_of[NCART_MAX];
        int keys[4], nk = 0;
        int k = 0;
        for (int i = 0; i <= l; ++i)
            for (int j = 0; j <= i; ++j, ++k) {
                const int ax = l - i, ay = i - j, az = j;
                const int key = (ax & 1) | ((ay & 1) << 1) | ((az & 1) << 2);
                int c = 0;
                while (c < nk && keys[c] != key) ++c;
                if (c == nk) keys[nk++] = key;
                key_of[k] = c;
                T.comp[c][T.na[c]++] = ax | (ay << 8) | (az << 16);
            }
        T.ncls = nk;
        // each solid function's nonzero coefficients lie in exactly one class
        for (int m = 0; m < 2 * l + 1; ++m) {
            int cls = -1;
            for (int q = 0; q < nc; ++q)
                if (std::fabs(C[m * nc + q]) > 1e-14) cls = key_of[q];
            const int jm = T.nm[cls]++;
            T.mind[cls][jm] = m;
            for (int ia = 0; ia < T.na[cls]; ++ia) {
                // ordinal of the class member ia
                int q = 0, seen = 0;
                for (; q < nc; ++q)
                    if (key_of[q] == cls && seen++ == ia) break;
                T.c[cls][jm][ia] = C[m * nc + q];
            }
        }
    }
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
