/*
 * Reference (oracle) evaluation of 4-center electron-repulsion integrals (ab|cd)
 * by the McMurchie-Davidson scheme, written plainly in FP64.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the CPU oracle that the CUDA path is
 * checked against.  Only the test-suite, the smoke check and the CPU-baseline leg
 * of the benchmark may load it.  It shares no code, header, table or constant
 * generator with the CUDA library, and it never calls that library.
 *
 * Steps follow the paper's Section 2 (Formalism) in the paper's order:
 *   1. Gaussian product: zeta_p = zeta_a + zeta_b, R_p = (zeta_a R_a + zeta_b R_b)/zeta_p
 *      (text after Eq. cart2herm-2).
 *   2. Hermite expansion coefficients (E_i)^t_{ab} by the two recursions printed after
 *      Eq. cart2herm-2, starting from (E_i)^0_{00} = 1; the Gaussian-product prefactor
 *      exp(-zeta_a zeta_b/zeta_p |AB|^2) that the printed start value leaves out is
 *      applied once per primitive pair.
 *   3. Boys function F_m(T) (Eq. boys) and [0]^(m) = (-2 rho)^m 2 pi^{5/2} /
 *      (zeta_p zeta_q sqrt(zeta_p + zeta_q)) F_m(rho |R_p - R_q|^2).
 *   4. Auxiliary Hermite integrals [r]^(m) by Eq. md1, from m = L down to 0.
 *   5. 2-index Hermite integrals [p|q] = (-1)^{l_q} [p+q]^(0) (Eq. pq).
 *   6. Bra transform [ab|q] = sum_p E_ab^p [p|q] (Eq. ab_to_hermite), then ket transform
 *      [ab|cd] = sum_q E_cd^q [ab|q] (Eq. cd_to_hermite), over Cartesian components.
 *   7. Contraction over primitives with normalised coefficients.
 *   8. Optional Cartesian-to-real-solid-harmonic transform, one index at a time
 *      (the coefficients C^a_{lm} of Section 2, Eq. for H; Schlegel & Frisch 1995).
 *
 * Conventions that the paper leaves open (recorded as readings in the design notes):
 *   - Cartesian order within a shell: for i = 0..l, j = 0..i: (l-i, i-j, j).
 *   - Each Cartesian primitive carries the normaliser of x^l:
 *       N(zeta, l) = (2 zeta/pi)^{3/4} (4 zeta)^{l/2} / sqrt((2l-1)!!).
 *   - A contracted shell is rescaled so that its x^l component has unit self-overlap.
 *   - Real solid harmonics are unit-normalised and ordered m = -l..l.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_LMAX 8                 /* largest shell angular momentum handled */
#define OR_LTOT (4 * OR_LMAX)     /* largest total angular momentum L */
#define OR_KMAX 64                /* largest contraction degree of one shell */

static const double OR_PI = 3.14159265358979323846264338327950288;

static int or_ncart(int l) { return (l + 1) * (l + 2) / 2; }

/* Cartesian exponents of component k of a shell with angular momentum l. */
static void or_cart(int l, int k, int *ax, int *ay, int *az)
{
    int n = 0;
    for (int i = 0; i <= l; ++i)
        for (int j = 0; j <= i; ++j) {
            if (n == k) { *ax = l - i; *ay = i - j; *az = j; return; }
            ++n;
        }
    *ax = *ay = *az = -1;
}

/* Number of Hermite triplets with t+u+v <= n (pyramidal number, Section 2 text). */
static int or_pyr(int n) { return (n + 1) * (n + 2) * (n + 3) / 6; }

/* Pyramidal ordinal of (t,u,v): all triplets of lower total n = t+u+v come first; within a
   total, i = u+v runs 0..n and v runs 0..i. */
static int or_pyr_index(int t, int u, int v)
{
    int n = t + u + v, i = u + v;
    return n * (n + 1) * (n + 2) / 6 + i * (i + 1) / 2 + v;
}

static void or_pyr_tuv(int idx, int *t, int *u, int *v)
{
    int n = 0;
    while (or_pyr(n) <= idx) ++n;
    int r = idx - (n > 0 ? or_pyr(n - 1) : 0);
    int i = 0;
    while ((i + 1) * (i + 2) / 2 <= r) ++i;
    *v = r - i * (i + 1) / 2;
    *u = i - *v;
    *t = n - i;
}

/* (2n-1)!! with (-1)!! = 1. */
static long double or_dfact_odd(int n)
{
    long double r = 1.0L;
    for (int k = 2 * n - 1; k > 1; k -= 2) r *= (long double)k;
    return r;
}

/* ------------------------------------------------------------------ Boys */

/*
 * F_m(T) = int_0^1 y^{2m} exp(-T y^2) dy  (Eq. boys), for m = 0..mmax.
 * For T <= 80 the convergent series
 *     F_m(T) = exp(-T) sum_k (2T)^k / [(2m+1)(2m+3)...(2m+2k+1)]
 * is summed in long double for m = mmax and the rest follows by the downward
 * recursion F_m = (2T F_{m+1} + exp(-T)) / (2m+1).  For T > 80, F_0 comes from
 * the error function, F_0 = (1/2) sqrt(pi/T) erf(sqrt T), and the upward recursion
 * F_{m+1} = ((2m+1) F_m - exp(-T)) / (2T) is used (its error factor (2m+1)/(2T)
 * stays below 1 for every m <= 2*OR_LTOT+1 < 160).
 */
void oracle_boys(int mmax, double T, double *F)
{
    long double t = (long double)T;
    long double e = expl(-t);
    if (T <= 80.0) {
        long double term = 1.0L / (2 * mmax + 1), sum = term;
        for (int k = 1; k < 100000; ++k) {
            term *= 2.0L * t / (long double)(2 * mmax + 2 * k + 1);
            sum += term;
            if (term < 1e-24L * sum && (long double)k > t) break;
        }
        long double f = e * sum;
        F[mmax] = (double)f;
        for (int m = mmax - 1; m >= 0; --m) {
            f = (2.0L * t * f + e) / (long double)(2 * m + 1);
            F[m] = (double)f;
        }
    } else {
        long double f = 0.5L * sqrtl(OR_PI / t) * erfl(sqrtl(t));
        F[0] = (double)f;
        for (int m = 0; m < mmax; ++m) {
            f = ((long double)(2 * m + 1) * f - e) / (2.0L * t);
            F[m + 1] = (double)f;
        }
    }
}

/* ------------------------------------------------------------ normalisation */

/* Normaliser of x^l exp(-zeta r^2): (2 zeta/pi)^{3/4} (4 zeta)^{l/2} / sqrt((2l-1)!!). */
double oracle_prim_norm(int l, double zeta)
{
    long double z = zeta;
    return (double)(powl(2.0L * z / OR_PI, 0.75L) * powl(4.0L * z, 0.5L * l) / sqrtl(or_dfact_odd(l)));
}

/*
 * Normalised contraction coefficients: c'_i = c_i N(zeta_i, l) s with s chosen so that
 * sum_ij c'_i c'_j <x^l e^{-zeta_i r^2} | x^l e^{-zeta_j r^2}> = 1, using
 * <x^l e^{-a r^2}|x^l e^{-b r^2}> = (2l-1)!! / (2(a+b))^l * (pi/(a+b))^{3/2}.
 */
void oracle_contract_norm(int l, int K, const double *zeta, const double *c, double *out)
{
    long double s = 0.0L;
    for (int i = 0; i < K; ++i)
        for (int j = 0; j < K; ++j) {
            long double ab = (long double)zeta[i] + zeta[j];
            long double ov = or_dfact_odd(l) / powl(2.0L * ab, l) * powl(OR_PI / ab, 1.5L);
            s += (long double)c[i] * c[j] * oracle_prim_norm(l, zeta[i]) * oracle_prim_norm(l, zeta[j]) * ov;
        }
    long double scale = 1.0L / sqrtl(s);
    for (int i = 0; i < K; ++i) out[i] = (double)(c[i] * oracle_prim_norm(l, zeta[i]) * scale);
}

/* ----------------------------------------------------------- solid harmonics */

static long double or_binom(int n, int k)
{
    if (k < 0 || k > n) return 0.0L;
    long double r = 1.0L;
    for (int i = 1; i <= k; ++i) r = r * (n - k + i) / i;
    return r;
}

/*
 * Real regular solid harmonics written out as Cartesian polynomials by the closed
 * form of Schlegel & Frisch (also Helgaker, Jorgensen & Olsen, Eq. 6.4.47-6.4.50):
 *   S_lm  ~ sum_{t=0}^{(l-|m|)/2} sum_{u=0}^{t} sum_{v} (-1)^{t+v-v_m} (1/4)^t
 *           C(l,t) C(l-t,|m|+t) C(t,u) C(|m|,2v) x^{2t+|m|-2(u+v)} y^{2(u+v)} z^{l-2t-|m|},
 * v_m = 0 (m >= 0) or 1/2 (m < 0), v running over v_m, v_m+1, ... up to floor(|m|/2 - v_m) + v_m.
 * Each polynomial is then scaled so that the solid Gaussian is unit-normalised when the
 * Cartesian functions carry the x^l normaliser; the result C[(m+l)*ncart + k] is the
 * coefficient of normalised Cartesian component k in unit-normalised solid function m.
 */
void oracle_solid_coefs(int l, double *C)
{
    int nc = or_ncart(l);
    for (int m = -l; m <= l; ++m) {
        long double poly[(OR_LMAX + 1) * (OR_LMAX + 2) / 2];
        for (int k = 0; k < nc; ++k) poly[k] = 0.0L;
        int am = m < 0 ? -m : m;
        int twovm = m < 0 ? 1 : 0; /* 2 v_m */
        for (int t = 0; t <= (l - am) / 2; ++t)
            for (int u = 0; u <= t; ++u)
                for (int k = 0; 2 * k + twovm <= am; ++k) { /* v - v_m = k, 2v = 2k + 2v_m */
                    int twov = 2 * k + twovm;
                    long double coef = ((t + k) % 2 ? -1.0L : 1.0L) * powl(0.25L, t) * or_binom(l, t) *
                                       or_binom(l - t, am + t) * or_binom(t, u) * or_binom(am, twov);
                    int px = 2 * t + am - 2 * u - twov, py = 2 * u + twov, pz = l - 2 * t - am;
                    if (px < 0) continue;
                    for (int q = 0; q < nc; ++q) {
                        int ax, ay, az;
                        or_cart(l, q, &ax, &ay, &az);
                        if (ax == px && ay == py && az == pz) { poly[q] += coef; break; }
                    }
                }
        /* <poly|poly> in units where <x^l|x^l> = (2l-1)!!:
           <x^a y^b z^c | x^a' y^b' z^c'> ∝ (a+a'-1)!! (b+b'-1)!! (c+c'-1)!! for even sums. */
        long double nrm = 0.0L;
        for (int p = 0; p < nc; ++p)
            for (int q = 0; q < nc; ++q) {
                int ax, ay, az, bx, by, bz;
                or_cart(l, p, &ax, &ay, &az);
                or_cart(l, q, &bx, &by, &bz);
                if ((ax + bx) % 2 || (ay + by) % 2 || (az + bz) % 2) continue;
                nrm += poly[p] * poly[q] * or_dfact_odd((ax + bx) / 2) * or_dfact_odd((ay + by) / 2) *
                       or_dfact_odd((az + bz) / 2);
            }
        long double s = sqrtl(or_dfact_odd(l) / nrm);
        for (int q = 0; q < nc; ++q) C[(m + l) * nc + q] = (double)(poly[q] * s);
    }
}

/* ------------------------------------------------------- Hermite expansion */

/*
 * 1-D Hermite expansion coefficients E[(i*(lb+1) + j)*(la+lb+1) + t] = (E_x)^t_{ij} for
 * i <= la, j <= lb, t <= la+lb, from the two recursions after Eq. cart2herm-2:
 *   E^t_{i+1,j} = E^{t-1}_{ij}/(2 zeta_p) + (P_x - A_x) E^t_{ij} + (t+1) E^{t+1}_{ij}
 *   E^t_{i,j+1} = E^{t-1}_{ij}/(2 zeta_p) + (P_x - B_x) E^t_{ij} + (t+1) E^{t+1}_{ij}
 * with E^0_{00} = 1 (no Gaussian-product factor here).
 */
void oracle_hermite_E(int la, int lb, double za, double zb, double Ax, double Bx, double *E)
{
    int nt = la + lb + 1;
    double zp = za + zb, Px = (za * Ax + zb * Bx) / zp;
    double PA = Px - Ax, PB = Px - Bx, oo2p = 1.0 / (2.0 * zp);
#define EI(i, j, t) E[((i) * (lb + 1) + (j)) * nt + (t)]
    for (int i = 0; i < (la + 1) * (lb + 1) * nt; ++i) E[i] = 0.0;
    EI(0, 0, 0) = 1.0;
    for (int i = 0; i <= la; ++i) {
        if (i > 0)
            for (int t = 0; t <= i; ++t) {
                double v = PA * EI(i - 1, 0, t);
                if (t > 0) v += oo2p * EI(i - 1, 0, t - 1);
                if (t + 1 <= i - 1) v += (t + 1) * EI(i - 1, 0, t + 1);
                EI(i, 0, t) = v;
            }
        for (int j = 1; j <= lb; ++j)
            for (int t = 0; t <= i + j; ++t) {
                double v = 0.0;
                if (t <= i + j - 1) v += PB * EI(i, j - 1, t);
                if (t > 0) v += oo2p * EI(i, j - 1, t - 1);
                if (t + 1 <= i + j - 1) v += (t + 1) * EI(i, j - 1, t + 1);
                EI(i, j, t) = v;
            }
    }
#undef EI
}

/* -------------------------------------------------------- Hermite integrals */

/*
 * Auxiliary integrals [r]^(0) for all |r| <= L (Eq. md1) for one primitive quartet:
 * R[(t*(L+1) + u)*(L+1) + v] for t+u+v <= L.  Inputs: rho, PQ = R_p - R_q, and the
 * prefactor pref = 2 pi^{5/2}/(zeta_p zeta_q sqrt(zeta_p+zeta_q)).
 * Work array: (L+1)^4 doubles.
 */
void oracle_hermite_R(int L, double rho, const double *PQ, double pref, double *R, double *work)
{
    int n1 = L + 1;
    double F[2 * OR_LTOT + 2];
    double T = rho * (PQ[0] * PQ[0] + PQ[1] * PQ[1] + PQ[2] * PQ[2]);
    oracle_boys(L, T, F);
#define RM(m, t, u, v) work[(((size_t)(m) * n1 + (t)) * n1 + (u)) * n1 + (v)]
    for (int m = L; m >= 0; --m) {
        RM(m, 0, 0, 0) = pow(-2.0 * rho, m) * pref * F[m];
        for (int n = 1; n <= L - m; ++n)
            for (int t = 0; t <= n; ++t)
                for (int u = 0; u <= n - t; ++u) {
                    int v = n - t - u;
                    double val;
                    /* [r + 1_i]^(m) = r_i [r - 1_i]^(m+1) + (P_i - Q_i) [r]^(m+1) */
                    if (t > 0) {
                        val = PQ[0] * RM(m + 1, t - 1, u, v);
                        if (t > 1) val += (t - 1) * RM(m + 1, t - 2, u, v);
                    } else if (u > 0) {
                        val = PQ[1] * RM(m + 1, t, u - 1, v);
                        if (u > 1) val += (u - 1) * RM(m + 1, t, u - 2, v);
                    } else {
                        val = PQ[2] * RM(m + 1, t, u, v - 1);
                        if (v > 1) val += (v - 1) * RM(m + 1, t, u, v - 2);
                    }
                    RM(m, t, u, v) = val;
                }
    }
    for (int t = 0; t <= L; ++t)
        for (int u = 0; u + t <= L; ++u)
            for (int v = 0; v + u + t <= L; ++v) R[(t * n1 + u) * n1 + v] = RM(0, t, u, v);
#undef RM
}

/* ------------------------------------------------------------ shell quartet */

typedef struct {
    double *E1[3], *E2[3]; /* 1-D E tables of bra and ket */
    double *Rw, *R0;       /* Eq. md1 work, [r]^(0) */
    double *pq;            /* [p|q] */
    double *abq;           /* [ab|q] */
    double *prim;          /* primitive Cartesian [ab|cd] */
    double *cart;          /* contracted Cartesian (ab|cd) */
    double *tmp1, *tmp2;   /* solid transform */
} or_scratch;

static void or_scratch_alloc(or_scratch *s, int lmax)
{
    int L = 4 * lmax, n1 = L + 1, lb = 2 * lmax, nt = lb + 1;
    int nherm = or_pyr(lb); /* Hermite triplets of one side */
    int nc = or_ncart(lmax), nab = nc * nc;
    for (int i = 0; i < 3; ++i) {
        s->E1[i] = malloc(sizeof(double) * (lmax + 1) * (lmax + 1) * nt);
        s->E2[i] = malloc(sizeof(double) * (lmax + 1) * (lmax + 1) * nt);
    }
    s->Rw = malloc(sizeof(double) * (size_t)n1 * n1 * n1 * n1);
    s->R0 = malloc(sizeof(double) * (size_t)n1 * n1 * n1);
    s->pq = malloc(sizeof(double) * (size_t)nherm * nherm);
    s->abq = malloc(sizeof(double) * (size_t)nab * nherm);
    s->prim = malloc(sizeof(double) * (size_t)nab * nab);
    s->cart = malloc(sizeof(double) * (size_t)nab * nab);
    s->tmp1 = malloc(sizeof(double) * (size_t)nab * nab);
    s->tmp2 = malloc(sizeof(double) * (size_t)nab * nab);
}

static void or_scratch_free(or_scratch *s)
{
    for (int i = 0; i < 3; ++i) { free(s->E1[i]); free(s->E2[i]); }
    free(s->Rw); free(s->R0); free(s->pq); free(s->abq); free(s->prim); free(s->cart);
    free(s->tmp1); free(s->tmp2);
}

/* One-index solid transform of index `which` (0..3) of a 4-index block with dims d[4]:
   out[..., m, ...] = sum_k C[m][k] in[..., k, ...]; updates d[which] to 2l+1. */
static void or_solid_one_index(const double *in, double *out, int *d, int which, int l)
{
    int nc = or_ncart(l), ns = 2 * l + 1;
    double C[(2 * OR_LMAX + 1) * ((OR_LMAX + 1) * (OR_LMAX + 2) / 2)];
    oracle_solid_coefs(l, C);
    size_t outer = 1, inner = 1;
    for (int i = 0; i < which; ++i) outer *= d[i];
    for (int i = which + 1; i < 4; ++i) inner *= d[i];
    for (size_t o = 0; o < outer; ++o)
        for (int m = 0; m < ns; ++m)
            for (size_t in_ = 0; in_ < inner; ++in_) {
                double acc = 0.0;
                for (int k = 0; k < nc; ++k) acc += C[m * nc + k] * in[(o * nc + k) * inner + in_];
                out[(o * ns + m) * inner + in_] = acc;
            }
    d[which] = ns;
}

typedef struct {
    int l, K;
    const double *zeta, *coef; /* coef already normalised (or raw) */
    double A[3];
} or_shell;

/* Contracted Cartesian (ab|cd) of one shell quartet by Steps 1-7; result in s->cart. */
static void or_quartet_md(const or_shell *sa, const or_shell *sb, const or_shell *sc, const or_shell *sd,
                          or_scratch *s)
{
    int la = sa->l, lb = sb->l, lc = sc->l, ld = sd->l;
    int lbra = la + lb, lket = lc + ld, L = lbra + lket, n1 = L + 1;
    int nta = lbra + 1, ntc = lket + 1;
    int na = or_ncart(la), nb = or_ncart(lb), nc = or_ncart(lc), nd = or_ncart(ld);
    int nab = na * nb, ncd = nc * nd;
    for (int i = 0; i < nab * ncd; ++i) s->cart[i] = 0.0;

    for (int ia = 0; ia < sa->K; ++ia)
        for (int ib = 0; ib < sb->K; ++ib) {
            double za = sa->zeta[ia], zb = sb->zeta[ib], zp = za + zb;
            double P[3], AB2 = 0.0;
            for (int x = 0; x < 3; ++x) {
                P[x] = (za * sa->A[x] + zb * sb->A[x]) / zp;
                AB2 += (sa->A[x] - sb->A[x]) * (sa->A[x] - sb->A[x]);
            }
            double Kab = exp(-za * zb / zp * AB2) * sa->coef[ia] * sb->coef[ib];
            for (int x = 0; x < 3; ++x) oracle_hermite_E(la, lb, za, zb, sa->A[x], sb->A[x], s->E1[x]);
            for (int ic = 0; ic < sc->K; ++ic)
                for (int id = 0; id < sd->K; ++id) {
                    double zc = sc->zeta[ic], zd = sd->zeta[id], zq = zc + zd;
                    double Q[3], CD2 = 0.0, PQ[3];
                    for (int x = 0; x < 3; ++x) {
                        Q[x] = (zc * sc->A[x] + zd * sd->A[x]) / zq;
                        CD2 += (sc->A[x] - sd->A[x]) * (sc->A[x] - sd->A[x]);
                    }
                    for (int x = 0; x < 3; ++x) PQ[x] = P[x] - Q[x];
                    double Kcd = exp(-zc * zd / zq * CD2) * sc->coef[ic] * sd->coef[id];
                    for (int x = 0; x < 3; ++x) oracle_hermite_E(lc, ld, zc, zd, sc->A[x], sd->A[x], s->E2[x]);
                    double rho = zp * zq / (zp + zq);
                    double pref = 2.0 * pow(OR_PI, 2.5) / (zp * zq * sqrt(zp + zq));
                    oracle_hermite_R(L, rho, PQ, pref, s->R0, s->Rw);
                    /* Step 5, Eq. pq: [p|q] = (-1)^{|q|} [p+q]^(0) for |p| <= lbra, |q| <= lket
                       (p and q stored in pyramidal order, see or_pyr_index). */
                    int np_ = or_pyr(lbra), nq_ = or_pyr(lket);
                    for (int ip = 0; ip < np_; ++ip) {
                        int px, py, pz;
                        or_pyr_tuv(ip, &px, &py, &pz);
                        for (int iq = 0; iq < nq_; ++iq) {
                            int qx, qy, qz;
                            or_pyr_tuv(iq, &qx, &qy, &qz);
                            double sgn = ((qx + qy + qz) % 2) ? -1.0 : 1.0;
                            s->pq[(size_t)ip * nq_ + iq] = sgn * s->R0[((px + qx) * n1 + (py + qy)) * n1 + (pz + qz)];
                        }
                    }
                    /* Step 6a, Eq. ab_to_hermite: [ab|q] = sum_p E_ab^p [p|q]; E_ab^p vanishes unless
                       p_i <= a_i + b_i, which is the natural range of the sums in Eq. cart2herm-2. */
                    for (int a = 0; a < na; ++a)
                        for (int b = 0; b < nb; ++b) {
                            int ax, ay, az, bx, by, bz;
                            or_cart(la, a, &ax, &ay, &az);
                            or_cart(lb, b, &bx, &by, &bz);
                            double *row = s->abq + (size_t)(a * nb + b) * nq_;
                            for (int iq = 0; iq < nq_; ++iq) row[iq] = 0.0;
                            for (int px = 0; px <= ax + bx; ++px) {
                                double ex = s->E1[0][(ax * (lb + 1) + bx) * nta + px];
                                for (int py = 0; py <= ay + by; ++py) {
                                    double ey = s->E1[1][(ay * (lb + 1) + by) * nta + py];
                                    for (int pz = 0; pz <= az + bz; ++pz) {
                                        double ez = s->E1[2][(az * (lb + 1) + bz) * nta + pz];
                                        double e = ex * ey * ez;
                                        const double *pr = s->pq + (size_t)or_pyr_index(px, py, pz) * nq_;
                                        for (int iq = 0; iq < nq_; ++iq) row[iq] += e * pr[iq];
                                    }
                                }
                            }
                        }
                    /* Step 6b, Eq. cd_to_hermite: [ab|cd] = sum_q E_cd^q [ab|q]. */
                    for (int c = 0; c < nc; ++c)
                        for (int d = 0; d < nd; ++d) {
                            int cx, cy, cz, dx, dy, dz;
                            or_cart(lc, c, &cx, &cy, &cz);
                            or_cart(ld, d, &dx, &dy, &dz);
                            for (int ab = 0; ab < nab; ++ab) {
                                const double *row = s->abq + (size_t)ab * nq_;
                                double acc = 0.0;
                                for (int qx = 0; qx <= cx + dx; ++qx) {
                                    double ex = s->E2[0][(cx * (ld + 1) + dx) * ntc + qx];
                                    for (int qy = 0; qy <= cy + dy; ++qy) {
                                        double ey = s->E2[1][(cy * (ld + 1) + dy) * ntc + qy];
                                        for (int qz = 0; qz <= cz + dz; ++qz) {
                                            double ez = s->E2[2][(cz * (ld + 1) + dz) * ntc + qz];
                                            acc += ex * ey * ez * row[or_pyr_index(qx, qy, qz)];
                                        }
                                    }
                                }
                                s->prim[(size_t)ab * ncd + c * nd + d] = acc;
                            }
                        }
                    /* Step 7: contraction. */
                    double f = Kab * Kcd;
                    for (int i = 0; i < nab * ncd; ++i) s->cart[i] += f * s->prim[i];
                }
        }
}

/* Contracted Cartesian (ab|cd) by the Obara-Saika / Head-Gordon-Pople route (eri_os_oracle.c). */
void oracle_os_quartet_cart(int la, int lb, int lc, int ld, const double *A, const double *B, const double *C,
                            const double *D, int Ka, int Kb, int Kc, int Kd, const double *za, const double *zb,
                            const double *zc, const double *zd, const double *ca, const double *cb,
                            const double *cc, const double *cd, double *out);

/*
 * Batch driver.  Shell s: angular momentum shell_l[s], shell_nprim[s] primitives starting at
 * shell_prim_off[s] in exps/coefs, center centers[3s..3s+2].  Quartet q: shells
 * quartet_shells[4q..4q+3], output block at out + out_off[q], row-major over the (a,b,c,d)
 * components.  solid != 0 gives real solid harmonics; normalize != 0 applies the conventions in
 * the file header, normalize == 0 uses the raw coefficients on unnormalised primitives.
 * method 0 = McMurchie-Davidson (this file), 1 = Obara-Saika/HGP (independent check).
 * Returns 0, or -1 on an invalid argument.
 */
int oracle_eri(int nshell, const int *shell_l, const int *shell_nprim, const int *shell_prim_off,
               const double *centers, const double *exps, const double *coefs, int64_t nquartet,
               const int *quartet_shells, const int64_t *out_off, int solid, int normalize, int method,
               int nthreads, double *out)
{
    int lmax = 0;
    for (int s = 0; s < nshell; ++s) {
        if (shell_l[s] < 0 || shell_l[s] > OR_LMAX || shell_nprim[s] < 1 || shell_nprim[s] > OR_KMAX) return -1;
        if (shell_l[s] > lmax) lmax = shell_l[s];
    }
    for (int64_t q = 0; q < 4 * nquartet; ++q)
        if (quartet_shells[q] < 0 || quartet_shells[q] >= nshell) return -1;
    /* normalised coefficients per shell */
    int nprim_tot = 0;
    for (int s = 0; s < nshell; ++s)
        if (shell_prim_off[s] + shell_nprim[s] > nprim_tot) nprim_tot = shell_prim_off[s] + shell_nprim[s];
    double *ncoef = malloc(sizeof(double) * (size_t)nshell * OR_KMAX);
    for (int s = 0; s < nshell; ++s) {
        const double *z = exps + shell_prim_off[s], *c = coefs + shell_prim_off[s];
        if (normalize) oracle_contract_norm(shell_l[s], shell_nprim[s], z, c, ncoef + (size_t)s * OR_KMAX);
        else for (int k = 0; k < shell_nprim[s]; ++k) ncoef[(size_t)s * OR_KMAX + k] = c[k];
    }
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
#pragma omp parallel
    {
        or_scratch scr;
        or_scratch_alloc(&scr, lmax);
#pragma omp for schedule(dynamic, 1)
        for (int64_t q = 0; q < nquartet; ++q) {
            or_shell sh[4];
            for (int k = 0; k < 4; ++k) {
                int s = quartet_shells[4 * q + k];
                sh[k].l = shell_l[s];
                sh[k].K = shell_nprim[s];
                sh[k].zeta = exps + shell_prim_off[s];
                sh[k].coef = ncoef + (size_t)s * OR_KMAX;
                for (int x = 0; x < 3; ++x) sh[k].A[x] = centers[3 * s + x];
            }
            if (method == 0) {
                or_quartet_md(&sh[0], &sh[1], &sh[2], &sh[3], &scr);
            } else {
                oracle_os_quartet_cart(sh[0].l, sh[1].l, sh[2].l, sh[3].l, sh[0].A, sh[1].A, sh[2].A, sh[3].A,
                                       sh[0].K, sh[1].K, sh[2].K, sh[3].K, sh[0].zeta, sh[1].zeta, sh[2].zeta,
                                       sh[3].zeta, sh[0].coef, sh[1].coef, sh[2].coef, sh[3].coef, scr.cart);
            }
            int d[4] = {or_ncart(sh[0].l), or_ncart(sh[1].l), or_ncart(sh[2].l), or_ncart(sh[3].l)};
            size_t n = (size_t)d[0] * d[1] * d[2] * d[3];
            if (!solid) {
                memcpy(out + out_off[q], scr.cart, n * sizeof(double));
            } else {
                or_solid_one_index(scr.cart, scr.tmp1, d, 0, sh[0].l);
                or_solid_one_index(scr.tmp1, scr.tmp2, d, 1, sh[1].l);
                or_solid_one_index(scr.tmp2, scr.tmp1, d, 2, sh[2].l);
                or_solid_one_index(scr.tmp1, scr.tmp2, d, 3, sh[3].l);
                memcpy(out + out_off[q], scr.tmp2, sizeof(double) * (size_t)d[0] * d[1] * d[2] * d[3]);
            }
        }
        or_scratch_free(&scr);
    }
    free(ncoef);
    return 0;
}

/* Threads the OpenMP runtime will use for a parallel region (for the CPU-baseline record). */
int oracle_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
