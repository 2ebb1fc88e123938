/*
 * Independent check evaluator for contracted Cartesian (ab|cd): the Obara-Saika vertical
 * recursion followed by the Head-Gordon-Pople horizontal recursion.
 *
 * TEST INFRASTRUCTURE ONLY (part of the oracle).  It exists to pin the plain
 * McMurchie-Davidson oracle with a second, algebraically different route to the same
 * integrals: a wrong sign, index or dropped term in either one shows up as a mismatch.
 * The paper names Obara-Saika (Head-Gordon-Pople variant) as the scheme of its CPU
 * comparison library (Section 1 and Section 4).
 *
 * Formulas (Obara & Saika 1986; Head-Gordon & Pople 1988), for primitives with
 * zeta = zeta_a + zeta_b, eta = zeta_c + zeta_d, W = (zeta P + eta Q)/(zeta + eta),
 * rho = zeta eta/(zeta + eta):
 *   (00|00)^(m) = 2 pi^{5/2} / (zeta eta sqrt(zeta+eta)) K_AB K_CD F_m(rho |PQ|^2)
 *   (e+1_i 0|f0)^(m) = PA_i (e0|f0)^(m) + WP_i (e0|f0)^(m+1)
 *        + e_i/(2 zeta) [(e-1_i 0|f0)^(m) - rho/zeta (e-1_i 0|f0)^(m+1)]
 *        + f_i/(2(zeta+eta)) (e0|f-1_i 0)^(m+1)
 *   (e0|f+1_i 0)^(m) = QC_i (e0|f0)^(m) + WQ_i (e0|f0)^(m+1)
 *        + f_i/(2 eta) [(e0|f-1_i 0)^(m) - rho/eta (e0|f-1_i 0)^(m+1)]
 *        + e_i/(2(zeta+eta)) (e-1_i 0|f0)^(m+1)
 *   (a, b+1_i| = (a+1_i, b| + (A_i - B_i) (a b|,   |c, d+1_i) = |c+1_i, d) + (C_i - D_i) |c d).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

void oracle_boys(int mmax, double T, double *F);

static const double OS_PI = 3.14159265358979323846264338327950288;

static int os_pyr(int n) { return n < 0 ? 0 : (n + 1) * (n + 2) * (n + 3) / 6; }
static int os_nc(int l) { return (l + 1) * (l + 2) / 2; }

/* Ordinal of (x,y,z) among all triplets of total <= n: lower totals first, then within
   the total n: i = y+z ascending, z ascending (the shell's Cartesian order). */
static int os_idx(int x, int y, int z)
{
    int n = x + y + z, i = y + z;
    return os_pyr(n - 1) + i * (i + 1) / 2 + z;
}

static void os_xyz(int idx, int *x, int *y, int *z)
{
    int n = 0;
    while (os_pyr(n) <= idx) ++n;
    int r = idx - os_pyr(n - 1), i = 0;
    while ((i + 1) * (i + 2) / 2 <= r) ++i;
    *z = r - i * (i + 1) / 2;
    *y = i - *z;
    *x = n - i;
}

/* Component k of shell l in the Cartesian order. */
static void os_comp(int l, int k, int c[3])
{
    int i = 0;
    while ((i + 1) * (i + 2) / 2 <= k) ++i;
    c[2] = k - i * (i + 1) / 2;
    c[1] = i - c[2];
    c[0] = l - i;
}

void oracle_os_quartet_cart(int la, int lb, int lc, int ld, const double *A, const double *B, const double *C,
                            const double *D, int Ka, int Kb, int Kc, int Kd, const double *za, const double *zb,
                            const double *zc, const double *zd, const double *ca, const double *cb,
                            const double *cc, const double *cd, double *out)
{
    const int lbra = la + lb, lket = lc + ld, L = lbra + lket, M = L + 1;
    const int ne = os_pyr(lbra), nf = os_pyr(lket);
    double *V = malloc(sizeof(double) * (size_t)ne * nf * M);       /* V[(f*ne + e)*M + m] */
    double *acc = calloc((size_t)ne * nf, sizeof(double));          /* contracted (e0|f0) */
    double F[4 * 8 + 2];
#define VV(f, e, m) V[((size_t)(f) * ne + (e)) * M + (m)]

    for (int ia = 0; ia < Ka; ++ia)
        for (int ib = 0; ib < Kb; ++ib)
            for (int ic = 0; ic < Kc; ++ic)
                for (int id = 0; id < Kd; ++id) {
                    double a = za[ia], b = zb[ib], c = zc[ic], d = zd[id];
                    double zeta = a + b, eta = c + d, rho = zeta * eta / (zeta + eta);
                    double P[3], Q[3], W[3], PA[3], WP[3], QC[3], WQ[3], AB2 = 0, CD2 = 0, PQ2 = 0;
                    for (int x = 0; x < 3; ++x) {
                        P[x] = (a * A[x] + b * B[x]) / zeta;
                        Q[x] = (c * C[x] + d * D[x]) / eta;
                        W[x] = (zeta * P[x] + eta * Q[x]) / (zeta + eta);
                        PA[x] = P[x] - A[x];
                        WP[x] = W[x] - P[x];
                        QC[x] = Q[x] - C[x];
                        WQ[x] = W[x] - Q[x];
                        AB2 += (A[x] - B[x]) * (A[x] - B[x]);
                        CD2 += (C[x] - D[x]) * (C[x] - D[x]);
                        PQ2 += (P[x] - Q[x]) * (P[x] - Q[x]);
                    }
                    double base = 2.0 * pow(OS_PI, 2.5) / (zeta * eta * sqrt(zeta + eta)) *
                                  exp(-a * b / zeta * AB2) * exp(-c * d / eta * CD2);
                    oracle_boys(L, rho * PQ2, F);
                    for (int m = 0; m <= L; ++m) VV(0, 0, m) = base * F[m];
                    /* bra VRR with f = 0 */
                    for (int e = 1; e < ne; ++e) {
                        int q[3];
                        os_xyz(e, &q[0], &q[1], &q[2]);
                        int i = q[0] ? 0 : (q[1] ? 1 : 2);
                        int qm[3] = {q[0], q[1], q[2]};
                        qm[i] -= 1;
                        int e1 = os_idx(qm[0], qm[1], qm[2]);
                        int n = q[0] + q[1] + q[2];
                        int e2 = -1;
                        if (qm[i] > 0) {
                            int q2[3] = {qm[0], qm[1], qm[2]};
                            q2[i] -= 1;
                            e2 = os_idx(q2[0], q2[1], q2[2]);
                        }
                        for (int m = 0; m <= L - n; ++m) {
                            double v = PA[i] * VV(0, e1, m) + WP[i] * VV(0, e1, m + 1);
                            if (e2 >= 0) v += qm[i] / (2.0 * zeta) * (VV(0, e2, m) - rho / zeta * VV(0, e2, m + 1));
                            VV(0, e, m) = v;
                        }
                    }
                    /* ket VRR */
                    for (int f = 1; f < nf; ++f) {
                        int r[3];
                        os_xyz(f, &r[0], &r[1], &r[2]);
                        int i = r[0] ? 0 : (r[1] ? 1 : 2);
                        int rm[3] = {r[0], r[1], r[2]};
                        rm[i] -= 1;
                        int f1 = os_idx(rm[0], rm[1], rm[2]);
                        int nfv = r[0] + r[1] + r[2];
                        int f2 = -1;
                        if (rm[i] > 0) {
                            int r2[3] = {rm[0], rm[1], rm[2]};
                            r2[i] -= 1;
                            f2 = os_idx(r2[0], r2[1], r2[2]);
                        }
                        for (int e = 0; e < ne; ++e) {
                            int q[3];
                            os_xyz(e, &q[0], &q[1], &q[2]);
                            int n = q[0] + q[1] + q[2];
                            int em = -1;
                            if (q[i] > 0) {
                                int qq[3] = {q[0], q[1], q[2]};
                                qq[i] -= 1;
                                em = os_idx(qq[0], qq[1], qq[2]);
                            }
                            for (int m = 0; m <= L - n - nfv; ++m) {
                                double v = QC[i] * VV(f1, e, m) + WQ[i] * VV(f1, e, m + 1);
                                if (f2 >= 0) v += rm[i] / (2.0 * eta) * (VV(f2, e, m) - rho / eta * VV(f2, e, m + 1));
                                if (em >= 0) v += q[i] / (2.0 * (zeta + eta)) * VV(f1, em, m + 1);
                                VV(f, e, m) = v;
                            }
                        }
                    }
                    double w = ca[ia] * cb[ib] * cc[ic] * cd[id];
                    for (int f = os_pyr(lc - 1); f < nf; ++f)
                        for (int e = os_pyr(la - 1); e < ne; ++e) acc[(size_t)e * nf + f] += w * VV(f, e, 0);
                }
#undef VV
    free(V);

    /* Bra HRR: level k holds (a, b| for |b| = k and la <= |a| <= lbra - k, each a row of nf. */
    const int f0 = os_pyr(lc - 1), nfr = nf - f0; /* ket rows used: lc <= |f| <= lket */
    const int a0 = os_pyr(la - 1);
    double *cur = malloc(sizeof(double) * (size_t)(ne - a0) * nfr);
    for (int e = a0; e < ne; ++e) memcpy(cur + (size_t)(e - a0) * nfr, acc + (size_t)e * nf + f0, sizeof(double) * nfr);
    free(acc);
    for (int k = 1; k <= lb; ++k) {
        int na_hi = os_pyr(lbra - k); /* a in [a0, na_hi) */
        int nbk = os_nc(k), nbk1 = os_nc(k - 1);
        double *nxt = malloc(sizeof(double) * (size_t)(na_hi - a0) * nbk * nfr);
        for (int ai = a0; ai < na_hi; ++ai) {
            int ax, ay, az;
            os_xyz(ai, &ax, &ay, &az);
            for (int bi = 0; bi < nbk; ++bi) {
                int bc[3];
                os_comp(k, bi, bc);
                int i = bc[0] ? 0 : (bc[1] ? 1 : 2);
                int bm[3] = {bc[0], bc[1], bc[2]};
                bm[i] -= 1;
                int bprev = os_idx(bm[0], bm[1], bm[2]) - os_pyr(k - 2); /* component within shell k-1 */
                int ap[3] = {ax, ay, az};
                ap[i] += 1;
                int aup = os_idx(ap[0], ap[1], ap[2]);
                const double *r1 = cur + ((size_t)(aup - a0) * nbk1 + bprev) * nfr;
                const double *r2 = cur + ((size_t)(ai - a0) * nbk1 + bprev) * nfr;
                double *o = nxt + ((size_t)(ai - a0) * nbk + bi) * nfr;
                double ABi = A[i] - B[i];
                for (int f = 0; f < nfr; ++f) o[f] = r1[f] + ABi * r2[f];
            }
        }
        free(cur);
        cur = nxt;
    }
    /* cur now holds (a b| for |a| = la (rows a0 .. a0+nc(la)), |b| = lb, each over the ket rows. */
    const int na = os_nc(la), nb = os_nc(lb), nc_ = os_nc(lc), nd = os_nc(ld);
    const int nab = na * nb;
    /* Ket HRR, same structure on the ket index, for each (ab). */
    const int c0 = f0;
    double *kc = malloc(sizeof(double) * (size_t)nab * nfr);
    memcpy(kc, cur, sizeof(double) * (size_t)nab * nfr);
    free(cur);
    for (int k = 1; k <= ld; ++k) {
        int nc_hi = os_pyr(lket - k);
        int ndk = os_nc(k), ndk1 = os_nc(k - 1);
        int ncur = nc_hi - c0;
        int nprev = os_pyr(lket - k + 1) - c0;
        double *nxt = malloc(sizeof(double) * (size_t)nab * ncur * ndk);
        for (int ab = 0; ab < nab; ++ab)
            for (int ci = c0; ci < nc_hi; ++ci) {
                int cx, cy, cz;
                os_xyz(ci, &cx, &cy, &cz);
                for (int di = 0; di < ndk; ++di) {
                    int dc[3];
                    os_comp(k, di, dc);
                    int i = dc[0] ? 0 : (dc[1] ? 1 : 2);
                    int dm[3] = {dc[0], dc[1], dc[2]};
                    dm[i] -= 1;
                    int dprev = os_idx(dm[0], dm[1], dm[2]) - os_pyr(k - 2);
                    int cp[3] = {cx, cy, cz};
                    cp[i] += 1;
                    int cup = os_idx(cp[0], cp[1], cp[2]);
                    double v1 = kc[((size_t)ab * nprev + (cup - c0)) * ndk1 + dprev];
                    double v2 = kc[((size_t)ab * nprev + (ci - c0)) * ndk1 + dprev];
                    nxt[((size_t)ab * ncur + (ci - c0)) * ndk + di] = v1 + (C[i] - D[i]) * v2;
                }
            }
        free(kc);
        kc = nxt;
    }
    /* kc holds (ab|c d) with c over rows [c0, c0 + nc(lc)) and d over shell ld. */
    for (int ab = 0; ab < nab; ++ab)
        for (int c = 0; c < nc_; ++c)
            for (int d = 0; d < nd; ++d) out[((size_t)ab * nc_ + c) * nd + d] = kc[((size_t)ab * nc_ + c) * nd + d];
    free(kc);
}
