/*
 * FP64 CPU oracle for the grouped generalized Coulomb / exchange builds.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path links, loads or
 * calls this file: only the tests, the smoke check and the benchmark's CPU
 * baseline leg use it.  It shares no code, header, table or helper with the
 * CUDA library; the two meet only in the seeded input generator.
 *
 * What it computes (plain definitions, no blocking or fusion):
 *   - contracted s-type Gaussians normalised to <phi|phi> = 1 (textbook,
 *     Szabo & Ostlund App. A, the text the paper cites for integrals);
 *   - primitive (ss|ss) integrals through the Boys function F0 closed form;
 *   - Cartesian p and d functions (labels 1..9) by the Obara-Saika vertical
 *     and Head-Gordon-Pople horizontal recurrences over F_0 .. F_8;
 *   - Schwarz factors Q_pq = sqrt((pq|pq));
 *   - generalized J, K and F of Eq. (J_and_K), Sec. II.B.1:
 *       J[D]_pq = sum_rs D_rs (rs|pq),  K[D]_pq = sum_rs D_rs (pr|qs),
 *       F = 2J - K,  for non-symmetric D;
 *   - the inner product D.F = sum_pq D_pq F_pq of Table I (notation table).
 * Screening reading: a quartet (pq|rs) is kept iff Q_pq * Q_rs >= tol
 * (tol = 0 keeps every quartet).  The paper's own rule (Sec. II.C) drops a
 * pair whose largest integral is below a threshold; the Schwarz product
 * rule is the bound-based form of the same idea.
 *
 * Every floating point operation is IEEE double.  erf() is the C library's.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_PI 3.14159265358979323846

/* offsets of each function's primitives in the flat exps / weights arrays */
static int64_t *prim_offsets(int n, const int32_t *nprim)
{
    int64_t *off = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n + 1));
    off[0] = 0;
    for (int i = 0; i < n; ++i) off[i + 1] = off[i] + nprim[i];
    return off;
}

/*
 * Normalisation (textbook): primitive g_k = (2 a_k / pi)^{3/4} exp(-a_k r^2)
 * has <g_k|g_k> = 1; <g_k|g_l> on one center = (2 sqrt(a_k a_l)/(a_k+a_l))^{3/2}.
 * phi = c sum_k d_k g_k with c chosen so that <phi|phi> = 1.
 * Output w_k = c d_k (2 a_k/pi)^{3/4}: the weight of the raw exp(-a_k r^2).
 */
int oracle_normalize(int n, const int32_t *nprim, const double *exps,
                     const double *coefs, double *w)
{
    if (n <= 0) return -1;
    int64_t *off = prim_offsets(n, nprim);
    for (int mu = 0; mu < n; ++mu) {
        double s = 0.0;
        for (int64_t k = off[mu]; k < off[mu + 1]; ++k)
            for (int64_t l = off[mu]; l < off[mu + 1]; ++l) {
                double ak = exps[k], al = exps[l];
                double ov = pow(2.0 * sqrt(ak * al) / (ak + al), 1.5);
                s += coefs[k] * coefs[l] * ov;
            }
        double c = 1.0 / sqrt(s);
        for (int64_t k = off[mu]; k < off[mu + 1]; ++k)
            w[k] = c * coefs[k] * pow(2.0 * exps[k] / OR_PI, 0.75);
    }
    free(off);
    return 0;
}

/* Boys function of order zero, F0(T) = int_0^1 exp(-T u^2) du
 *   = (1/2) sqrt(pi/T) erf(sqrt(T))  for T > 0, with the Taylor series
 *   sum_k (-T)^k / (k! (2k+1)) for small T (four terms below 1e-6). */
double oracle_boys0(double T)
{
    if (T < 1e-6) return 1.0 - T / 3.0 + T * T / 10.0 - T * T * T / 42.0;
    return 0.5 * sqrt(OR_PI / T) * erf(sqrt(T));
}

/* [ab|cd] over raw Gaussians exp(-a|r-A|^2) ... (textbook, Boys 1950):
 *   p = a+b, q = c+d, P = (aA+bB)/p, Q = (cC+dD)/q, rho = pq/(p+q)
 *   [ab|cd] = 2 pi^{5/2} / (p q sqrt(p+q)) exp(-ab/p |AB|^2)
 *             exp(-cd/q |CD|^2) F0(rho |PQ|^2) */
static double prim_eri(double a, const double *A, double b, const double *B,
                       double c, const double *C, double d, const double *D)
{
    double p = a + b, q = c + d;
    double P[3], Q[3], ab2 = 0, cd2 = 0, pq2 = 0;
    for (int x = 0; x < 3; ++x) {
        P[x] = (a * A[x] + b * B[x]) / p;
        Q[x] = (c * C[x] + d * D[x]) / q;
        ab2 += (A[x] - B[x]) * (A[x] - B[x]);
        cd2 += (C[x] - D[x]) * (C[x] - D[x]);
        pq2 += (P[x] - Q[x]) * (P[x] - Q[x]);
    }
    double T = p * q / (p + q) * pq2;
    return 2.0 * pow(OR_PI, 2.5) / (p * q * sqrt(p + q)) *
           exp(-a * b / p * ab2) * exp(-c * d / q * cd2) * oracle_boys0(T);
}

/*
 * Cartesian p and d functions (angular momentum 1 and 2).  A function's
 * Cartesian label cart = 0 (s), 1, 2, 3 (p_x, p_y, p_z), 4, 5, 6 (d_xx, d_yy,
 * d_zz), 7, 8, 9 (d_xy, d_xz, d_yz) makes its primitives
 * (x - A_x)^lx (y - A_y)^ly (z - A_z)^lz exp(-a |r - A|^2) with the exponent
 * triple (lx, ly, lz) of the label.  Integrals over them follow the Obara-Saika
 * recurrences (Obara & Saika, J. Chem. Phys. 84, 3963 (1986)): the vertical
 * recurrence builds [e0|f0]^(m) from the Boys functions F_m, the horizontal
 * one (Head-Gordon & Pople, J. Chem. Phys. 89, 5777 (1988)) moves angular
 * momentum from the first to the second function of a pair:
 *   [e+1_i 0|f0]^(m) = PA_i [e0|f0]^(m) + WP_i [e0|f0]^(m+1)
 *       + e_i/(2p) ([e-1_i 0|f0]^(m) - rho/p [e-1_i 0|f0]^(m+1))
 *       + f_i/(2(p+q)) [e0|f-1_i 0]^(m+1)
 *   [00|f+1_i 0]^(m) = QC_i [00|f0]^(m) + WQ_i [00|f0]^(m+1)
 *       + f_i/(2q) ([00|f-1_i 0]^(m) - rho/q [00|f-1_i 0]^(m+1))
 *   [a, b+1_j| = [a+1_j, b| + (A - B)_j [a, b|     (and the same for the ket)
 * with W = (pP + qQ)/(p + q), rho = pq/(p + q) and
 * [00|00]^(m) = 2 pi^{5/2}/(pq sqrt(p+q)) exp(-ab/p |AB|^2) exp(-cd/q |CD|^2) F_m(T).
 */

/* F_m(T) = int_0^1 u^{2m} exp(-T u^2) du for m <= mmax: the top order from
 * the positive series F_M(T) = exp(-T) sum_k (2T)^k / ((2M+1)(2M+3)...(2M+2k+1)),
 * then downward recursion F_{m-1} = (2T F_m + exp(-T)) / (2m - 1). */
static void boys_all(int mmax, double T, double *F)
{
    double term = 1.0 / (2 * mmax + 1), sum = term;
    for (int k = 1; k < 2000; ++k) {
        term *= 2.0 * T / (2 * mmax + 2 * k + 1);
        sum += term;
        if (term < 1e-17 * sum) break;
    }
    double e = exp(-T);
    F[mmax] = e * sum;
    for (int m = mmax; m > 0; --m) F[m - 1] = (2.0 * T * F[m] + e) / (2 * m - 1);
}

double oracle_boys(int m, double T)
{
    double F[32];
    if (m < 0 || m > 30) return 0.0;
    boys_all(m, T, F);
    return F[m];
}

typedef struct {
    double PA[3], WP[3], QC[3], WQ[3], p, q, rho, K, F[16];
    /* values of [e0|f0]^(m) already formed for this primitive quartet, over
     * the box e <= E, f <= G (componentwise), m <= L; NAN = not yet formed */
    int E[3], G[3], L;
    double *memo;
} osdata;

static int vrr_slot(const osdata *o, const int *e, const int *f, int m)
{
    int ie = (e[0] * (o->E[1] + 1) + e[1]) * (o->E[2] + 1) + e[2];
    int nf = (o->G[0] + 1) * (o->G[1] + 1) * (o->G[2] + 1);
    int jf = (f[0] * (o->G[1] + 1) + f[1]) * (o->G[2] + 1) + f[2];
    return (ie * nf + jf) * (o->L + 1) + m;
}

static double os_vrr_formed(const osdata *o, const int *e, const int *f, int m);

/* [e0|f0]^(m) by the vertical recurrence (e, f: Cartesian exponent triples);
 * each value is formed once per primitive quartet and kept in o->memo */
static double os_vrr(const osdata *o, const int *e, const int *f, int m)
{
    int k = vrr_slot(o, e, f, m);
    if (isnan(o->memo[k])) o->memo[k] = os_vrr_formed(o, e, f, m);
    return o->memo[k];
}

static double os_vrr_formed(const osdata *o, const int *e, const int *f, int m)
{
    int i;
    for (i = 0; i < 3 && e[i] == 0; ++i) {}
    if (i < 3) {
        int e1[3] = {e[0], e[1], e[2]};
        e1[i] -= 1;
        double v = o->PA[i] * os_vrr(o, e1, f, m) + o->WP[i] * os_vrr(o, e1, f, m + 1);
        if (e1[i] > 0) {
            int e2[3] = {e1[0], e1[1], e1[2]};
            e2[i] -= 1;
            v += e1[i] / (2.0 * o->p) * (os_vrr(o, e2, f, m) - o->rho / o->p * os_vrr(o, e2, f, m + 1));
        }
        if (f[i] > 0) {
            int f1[3] = {f[0], f[1], f[2]};
            f1[i] -= 1;
            v += f[i] / (2.0 * (o->p + o->q)) * os_vrr(o, e1, f1, m + 1);
        }
        return v;
    }
    for (i = 0; i < 3 && f[i] == 0; ++i) {}
    if (i == 3) return o->K * o->F[m];
    int f1[3] = {f[0], f[1], f[2]};
    f1[i] -= 1;
    double v = o->QC[i] * os_vrr(o, e, f1, m) + o->WQ[i] * os_vrr(o, e, f1, m + 1);
    if (f1[i] > 0) {
        int f2[3] = {f1[0], f1[1], f1[2]};
        f2[i] -= 1;
        v += f1[i] / (2.0 * o->q) * (os_vrr(o, e, f2, m) - o->rho / o->q * os_vrr(o, e, f2, m + 1));
    }
    return v;
}

/* [a b|c d] by the horizontal recurrence down to [e0|f0]^(0) */
static double os_hrr(const osdata *o, const double *AB, const double *CD,
                     const int *a, const int *b, const int *c, const int *d)
{
    int j;
    for (j = 0; j < 3 && b[j] == 0; ++j) {}
    if (j < 3) {
        int a1[3] = {a[0], a[1], a[2]}, b1[3] = {b[0], b[1], b[2]};
        a1[j] += 1;
        b1[j] -= 1;
        return os_hrr(o, AB, CD, a1, b1, c, d) + AB[j] * os_hrr(o, AB, CD, a, b1, c, d);
    }
    for (j = 0; j < 3 && d[j] == 0; ++j) {}
    if (j < 3) {
        int c1[3] = {c[0], c[1], c[2]}, d1[3] = {d[0], d[1], d[2]};
        c1[j] += 1;
        d1[j] -= 1;
        return os_hrr(o, AB, CD, a, b, c1, d1) + CD[j] * os_hrr(o, AB, CD, a, b, c, d1);
    }
    return os_vrr(o, a, c, 0);
}

/* exponent triple of a Cartesian label (0 s; 1-3 p_x, p_y, p_z; 4-6 d_xx,
 * d_yy, d_zz; 7-9 d_xy, d_xz, d_yz) */
static void cart_vec(int cart, int *v)
{
    static const int tab[10][3] = {{0, 0, 0}, {1, 0, 0}, {0, 1, 0}, {0, 0, 1}, {2, 0, 0},
                                   {0, 2, 0}, {0, 0, 2}, {1, 1, 0}, {1, 0, 1}, {0, 1, 1}};
    v[0] = tab[cart][0]; v[1] = tab[cart][1]; v[2] = tab[cart][2];
}

/* primitive [ab|cd] over raw Cartesian primitives with labels la..ld */
static double prim_eri_l(double a, const double *A, int la, double b, const double *B, int lb,
                         double c, const double *C, int lc, double d, const double *D, int ld)
{
    osdata o;
    double p = a + b, q = c + d, P[3], Q[3], W[3], AB[3], CD[3], ab2 = 0, cd2 = 0, pq2 = 0;
    for (int x = 0; x < 3; ++x) {
        P[x] = (a * A[x] + b * B[x]) / p;
        Q[x] = (c * C[x] + d * D[x]) / q;
        W[x] = (p * P[x] + q * Q[x]) / (p + q);
        AB[x] = A[x] - B[x];
        CD[x] = C[x] - D[x];
        ab2 += AB[x] * AB[x];
        cd2 += CD[x] * CD[x];
        pq2 += (P[x] - Q[x]) * (P[x] - Q[x]);
        o.PA[x] = P[x] - A[x];
        o.WP[x] = W[x] - P[x];
        o.QC[x] = Q[x] - C[x];
        o.WQ[x] = W[x] - Q[x];
    }
    o.p = p; o.q = q; o.rho = p * q / (p + q);
    o.K = 2.0 * pow(OR_PI, 2.5) / (p * q * sqrt(p + q)) * exp(-a * b / p * ab2) * exp(-c * d / q * cd2);
    int va[3], vb[3], vc[3], vd[3];
    cart_vec(la, va); cart_vec(lb, vb); cart_vec(lc, vc); cart_vec(ld, vd);
    /* the horizontal recurrence moves b onto a and d onto c, so the vertical
     * one needs e <= a + b and f <= c + d, and orders m <= |a+b| + |c+d| */
    int L = 0;
    for (int x = 0; x < 3; ++x) {
        o.E[x] = va[x] + vb[x];
        o.G[x] = vc[x] + vd[x];
        L += o.E[x] + o.G[x];
    }
    o.L = L;
    boys_all(L, o.rho * pq2, o.F);
    double memo[13 * 13 * 9];   /* |a+b|, |c+d| <= 4: at most 12 triples per box, L <= 8 */
    int nmemo = (o.E[0] + 1) * (o.E[1] + 1) * (o.E[2] + 1) * (o.G[0] + 1) * (o.G[1] + 1) * (o.G[2] + 1) * (L + 1);
    for (int k = 0; k < nmemo; ++k) memo[k] = NAN;
    o.memo = memo;
    return os_hrr(&o, AB, CD, va, vb, vc, vd);
}

typedef struct {
    int n;
    const double *center;
    const int32_t *nprim;
    const double *exps;
    const double *w;
    int64_t *off;
    const int32_t *cart;      /* NULL: every function is s */
} obasis;

static obasis mk_basis(int n, const double *center, const int32_t *nprim,
                       const double *exps, const double *w)
{
    obasis b;
    b.n = n; b.center = center; b.nprim = nprim; b.exps = exps; b.w = w;
    b.off = prim_offsets(n, nprim);
    b.cart = NULL;
    return b;
}

/* contracted (pq|rs): sum over all primitive products */
static double eri_c(const obasis *b, int p, int q, int r, int s)
{
    if (b->cart && (b->cart[p] || b->cart[q] || b->cart[r] || b->cart[s])) {
        double v = 0.0;
        for (int64_t i = b->off[p]; i < b->off[p + 1]; ++i)
            for (int64_t j = b->off[q]; j < b->off[q + 1]; ++j)
                for (int64_t k = b->off[r]; k < b->off[r + 1]; ++k)
                    for (int64_t l = b->off[s]; l < b->off[s + 1]; ++l)
                        v += b->w[i] * b->w[j] * b->w[k] * b->w[l] *
                             prim_eri_l(b->exps[i], b->center + 3 * p, b->cart[p],
                                        b->exps[j], b->center + 3 * q, b->cart[q],
                                        b->exps[k], b->center + 3 * r, b->cart[r],
                                        b->exps[l], b->center + 3 * s, b->cart[s]);
        return v;
    }
    double v = 0.0;
    for (int64_t i = b->off[p]; i < b->off[p + 1]; ++i)
        for (int64_t j = b->off[q]; j < b->off[q + 1]; ++j)
            for (int64_t k = b->off[r]; k < b->off[r + 1]; ++k)
                for (int64_t l = b->off[s]; l < b->off[s + 1]; ++l)
                    v += b->w[i] * b->w[j] * b->w[k] * b->w[l] *
                         prim_eri(b->exps[i], b->center + 3 * p,
                                  b->exps[j], b->center + 3 * q,
                                  b->exps[k], b->center + 3 * r,
                                  b->exps[l], b->center + 3 * s);
    return v;
}

double oracle_eri(int n, const double *center, const int32_t *nprim,
                  const double *exps, const double *w, int p, int q, int r, int s)
{
    obasis b = mk_basis(n, center, nprim, exps, w);
    double v = eri_c(&b, p, q, r, s);
    free(b.off);
    return v;
}

/* full N^4 tensor, element [((p N + q) N + r) N + s] = (pq|rs), no symmetry used */
int oracle_eri_tensor(int n, const double *center, const int32_t *nprim,
                      const double *exps, const double *w, double *out)
{
    obasis b = mk_basis(n, center, nprim, exps, w);
    for (int p = 0; p < n; ++p)
        for (int q = 0; q < n; ++q)
            for (int r = 0; r < n; ++r)
                for (int s = 0; s < n; ++s)
                    out[(((int64_t)p * n + q) * n + r) * n + s] = eri_c(&b, p, q, r, s);
    free(b.off);
    return 0;
}

/* Q[p N + q] = Q[q N + p] = sqrt((pq|pq)), evaluated once for p >= q */
int oracle_schwarz(int n, const double *center, const int32_t *nprim,
                   const double *exps, const double *w, double *Q)
{
    obasis b = mk_basis(n, center, nprim, exps, w);
    for (int p = 0; p < n; ++p)
        for (int q = 0; q <= p; ++q) {
            double v = eri_c(&b, p, q, p, q);
            Q[(int64_t)p * n + q] = sqrt(v > 0.0 ? v : 0.0);
            Q[(int64_t)q * n + p] = Q[(int64_t)p * n + q];
        }
    free(b.off);
    return 0;
}

/*
 * Pair screening as Sec. II.C states it: for every index pair (p, q) the
 * largest |(pq|rs)| over all pairs (r, s); a pair is discarded when that
 * maximum is at most the threshold.  Brute force over the unique quartets
 * (pq >= rs), each updating both of its pairs.  out[p N + q] = out[q N + p].
 */
int oracle_pair_max(int n, const double *center, const int32_t *nprim,
                    const double *exps, const double *w, double *out)
{
    obasis b = mk_basis(n, center, nprim, exps, w);
    for (int64_t i = 0; i < (int64_t)n * n; ++i) out[i] = 0.0;
    for (int p = 0; p < n; ++p)
        for (int q = 0; q <= p; ++q)
            for (int r = 0; r <= p; ++r)
                for (int s = 0; s <= r; ++s) {
                    if (r == p && s > q) continue;          /* pair(rs) <= pair(pq) */
                    const double v = fabs(eri_c(&b, p, q, r, s));
                    double *a1 = out + (int64_t)p * n + q, *a2 = out + (int64_t)r * n + s;
                    if (v > *a1) *a1 = v;
                    if (v > *a2) *a2 = v;
                }
    for (int p = 0; p < n; ++p)
        for (int q = 0; q < p; ++q) out[(int64_t)q * n + p] = out[(int64_t)p * n + q];
    free(b.off);
    return 0;
}

static int kept(const double *Q, int n, int p, int q, int r, int s, double tol)
{
    return Q[(int64_t)p * n + q] * Q[(int64_t)r * n + s] >= tol;
}

/*
 * Brute force over all ordered (p,q,r,s) with a precomputed full tensor:
 *   J[p][q] += D[r][s] (pq|rs),  K[p][r] += D[q][s] (pq|rs).
 * This is Eq. (J_and_K) with the dummy indices renamed.  J, K are zeroed.
 */
int oracle_jk_brute(int n, const double *eri, const double *Q, double tol,
                    int m, const double *D, double *J, double *K)
{
    int64_t nn = (int64_t)n * n;
    memset(J, 0, sizeof(double) * (size_t)(nn * m));
    memset(K, 0, sizeof(double) * (size_t)(nn * m));
    for (int p = 0; p < n; ++p)
        for (int q = 0; q < n; ++q)
            for (int r = 0; r < n; ++r)
                for (int s = 0; s < n; ++s) {
                    if (!kept(Q, n, p, q, r, s, tol)) continue;
                    double v = eri[(((int64_t)p * n + q) * n + r) * n + s];
                    for (int k = 0; k < m; ++k) {
                        const double *Dk = D + k * nn;
                        J[k * nn + (int64_t)p * n + q] += Dk[(int64_t)r * n + s] * v;
                        K[k * nn + (int64_t)p * n + r] += Dk[(int64_t)q * n + s] * v;
                    }
                }
    return 0;
}

/* pair index of (p >= q) */
static int64_t pidx(int p, int q) { return (int64_t)p * (p + 1) / 2 + q; }

/*
 * Unique-quartet loop: each integral with p >= q, r >= s, pair(pq) >=
 * pair(rs) is evaluated once and applied to every DISTINCT ordered tuple in
 * its permutation orbit (p,q,r,s) (q,p,r,s) (p,q,s,r) (q,p,s,r) (r,s,p,q)
 * (s,r,p,q) (r,s,q,p) (s,r,q,p), using the same ordered update as the brute
 * loop.  No degeneracy factors are needed.
 * Bra pairs pq in [pair_begin, pair_end) are processed (the full build is
 * [0, N(N+1)/2)); J and K are accumulated, NOT zeroed, so that partial
 * ranges can be summed.  If eri_list is non-NULL it supplies the integrals
 * in loop order (stored mode) instead of evaluating them.
 * Returns the number of kept unique quartets.
 */
static int64_t jk_unique_core(obasis b, const double *Q, double tol, int m, const double *D,
                              double *J, double *K, int64_t pair_begin, int64_t pair_end,
                              const double *eri_list);

int64_t oracle_jk_unique(int n, const double *center, const int32_t *nprim,
                         const double *exps, const double *w, const double *Q,
                         double tol, int m, const double *D, double *J, double *K,
                         int64_t pair_begin, int64_t pair_end,
                         const double *eri_list)
{
    return jk_unique_core(mk_basis(n, center, nprim, exps, w), Q, tol, m, D, J, K,
                          pair_begin, pair_end, eri_list);
}

/* oracle_jk_unique for a basis with Cartesian p functions */
int64_t oracle_jk_unique_l(int n, const double *center, const int32_t *nprim,
                           const double *exps, const double *w, const int32_t *cart,
                           const double *Q, double tol, int m, const double *D,
                           double *J, double *K, int64_t pair_begin, int64_t pair_end)
{
    obasis b = mk_basis(n, center, nprim, exps, w);
    b.cart = cart;
    return jk_unique_core(b, Q, tol, m, D, J, K, pair_begin, pair_end, NULL);
}

static int64_t jk_unique_core(obasis b, const double *Q, double tol, int m, const double *D,
                              double *J, double *K, int64_t pair_begin, int64_t pair_end,
                              const double *eri_list)
{
    int n = b.n;
    int64_t nn = (int64_t)n * n;
    int64_t nkept = 0, pos = 0;
    /* walk all bra pairs, skip those outside the range */
    for (int p = 0; p < n; ++p)
        for (int q = 0; q <= p; ++q) {
            int64_t pq = pidx(p, q);
            if (pq < pair_begin || pq >= pair_end) continue;
            for (int r = 0; r <= p; ++r)
                for (int s = 0; s <= r; ++s) {
                    int64_t rs = pidx(r, s);
                    if (rs > pq) continue;
                    if (!kept(Q, n, p, q, r, s, tol)) continue;
                    double v = eri_list ? eri_list[pos++] : eri_c(&b, p, q, r, s);
                    ++nkept;
                    int t[8][4] = {{p, q, r, s}, {q, p, r, s}, {p, q, s, r}, {q, p, s, r},
                                   {r, s, p, q}, {s, r, p, q}, {r, s, q, p}, {s, r, q, p}};
                    for (int a = 0; a < 8; ++a) {
                        int dup = 0;
                        for (int c = 0; c < a; ++c)
                            if (t[a][0] == t[c][0] && t[a][1] == t[c][1] &&
                                t[a][2] == t[c][2] && t[a][3] == t[c][3]) { dup = 1; break; }
                        if (dup) continue;
                        int i0 = t[a][0], i1 = t[a][1], i2 = t[a][2], i3 = t[a][3];
                        for (int k = 0; k < m; ++k) {
                            const double *Dk = D + k * nn;
                            J[k * nn + (int64_t)i0 * n + i1] += Dk[(int64_t)i2 * n + i3] * v;
                            K[k * nn + (int64_t)i0 * n + i2] += Dk[(int64_t)i1 * n + i3] * v;
                        }
                    }
                }
        }
    free(b.off);
    return nkept;
}

/*
 * Density weight of each index pair for density-weighted screening:
 * Wd[x][y] = max over k of max(|D_k[x][y]|, |D_k[y][x]|)  (symmetric).
 */
int oracle_density_weight(int n, int m, const double *D, double *Wd)
{
    int64_t nn = (int64_t)n * n;
    for (int x = 0; x < n; ++x)
        for (int y = 0; y < n; ++y) {
            double v = 0.0;
            for (int k = 0; k < m; ++k) {
                double a = fabs(D[k * nn + (int64_t)x * n + y]);
                double b = fabs(D[k * nn + (int64_t)y * n + x]);
                if (a > v) v = a;
                if (b > v) v = b;
            }
            Wd[(int64_t)x * n + y] = v;
        }
    return 0;
}

/*
 * Density-weighted screening: the unique-quartet loop of oracle_jk_unique in
 * which a Schwarz-kept quartet (Q_pq Q_rs >= tol) is also dropped when
 *   Q_pq Q_rs max(Wd[r][s], Wd[p][q], Wd[q][s], Wd[p][s], Wd[q][r], Wd[p][r]) < tol_d.
 * Every update of Eq. (J_and_K) that the quartet makes multiplies it by one
 * of those density elements (J: D_rs, D_pq and transposes; K: D_qs, D_ps,
 * D_qr, D_pr and transposes), and |(pq|rs)| <= Q_pq Q_rs, so each dropped
 * update is below tol_d in magnitude.  The weight is shared by all m
 * densities of the grouped build.  Full range; J, K zeroed first.  Returns
 * the number of kept unique quartets.
 */
int64_t oracle_jk_unique_dw(int n, const double *center, const int32_t *nprim,
                            const double *exps, const double *w, const double *Q,
                            double tol, double tol_d, int m, const double *D,
                            double *J, double *K)
{
    obasis b = mk_basis(n, center, nprim, exps, w);
    int64_t nn = (int64_t)n * n;
    double *Wd = (double *)malloc(sizeof(double) * (size_t)nn);
    oracle_density_weight(n, m, D, Wd);
    memset(J, 0, sizeof(double) * (size_t)(nn * m));
    memset(K, 0, sizeof(double) * (size_t)(nn * m));
    int64_t nkept = 0;
    for (int p = 0; p < n; ++p)
        for (int q = 0; q <= p; ++q)
            for (int r = 0; r <= p; ++r)
                for (int s = 0; s <= r; ++s) {
                    if (pidx(r, s) > pidx(p, q)) continue;
                    if (!kept(Q, n, p, q, r, s, tol)) continue;
                    double wt = Wd[(int64_t)r * n + s];
                    double c[5] = {Wd[(int64_t)p * n + q], Wd[(int64_t)q * n + s], Wd[(int64_t)p * n + s],
                                   Wd[(int64_t)q * n + r], Wd[(int64_t)p * n + r]};
                    for (int i = 0; i < 5; ++i) if (c[i] > wt) wt = c[i];
                    if (Q[(int64_t)p * n + q] * Q[(int64_t)r * n + s] * wt < tol_d) continue;
                    double v = eri_c(&b, p, q, r, s);
                    ++nkept;
                    int t[8][4] = {{p, q, r, s}, {q, p, r, s}, {p, q, s, r}, {q, p, s, r},
                                   {r, s, p, q}, {s, r, p, q}, {r, s, q, p}, {s, r, q, p}};
                    for (int a = 0; a < 8; ++a) {
                        int dup = 0;
                        for (int c2 = 0; c2 < a; ++c2)
                            if (t[a][0] == t[c2][0] && t[a][1] == t[c2][1] &&
                                t[a][2] == t[c2][2] && t[a][3] == t[c2][3]) { dup = 1; break; }
                        if (dup) continue;
                        int i0 = t[a][0], i1 = t[a][1], i2 = t[a][2], i3 = t[a][3];
                        for (int k = 0; k < m; ++k) {
                            const double *Dk = D + k * nn;
                            J[k * nn + (int64_t)i0 * n + i1] += Dk[(int64_t)i2 * n + i3] * v;
                            K[k * nn + (int64_t)i0 * n + i2] += Dk[(int64_t)i1 * n + i3] * v;
                        }
                    }
                }
    free(Wd);
    free(b.off);
    return nkept;
}

/* The kept unique integrals in the loop order of oracle_jk_unique over
 * [pair_begin, pair_end); returns how many were written (at most cap). */
int64_t oracle_unique_list(int n, const double *center, const int32_t *nprim,
                           const double *exps, const double *w, const double *Q,
                           double tol, int64_t pair_begin, int64_t pair_end,
                           double *out, int64_t cap)
{
    obasis b = mk_basis(n, center, nprim, exps, w);
    int64_t cnt = 0;
    for (int p = 0; p < n; ++p)
        for (int q = 0; q <= p; ++q) {
            int64_t pq = pidx(p, q);
            if (pq < pair_begin || pq >= pair_end) continue;
            for (int r = 0; r <= p; ++r)
                for (int s = 0; s <= r; ++s) {
                    if (pidx(r, s) > pq) continue;
                    if (!kept(Q, n, p, q, r, s, tol)) continue;
                    if (cnt < cap) out[cnt] = eri_c(&b, p, q, r, s);
                    ++cnt;
                }
        }
    free(b.off);
    return cnt;
}

/* number of kept unique quartets for a Schwarz table */
int64_t oracle_count_kept(int n, const double *Q, double tol)
{
    int64_t cnt = 0;
    for (int p = 0; p < n; ++p)
        for (int q = 0; q <= p; ++q)
            for (int r = 0; r <= p; ++r)
                for (int s = 0; s <= r; ++s)
                    if (pidx(r, s) <= pidx(p, q) && kept(Q, n, p, q, r, s, tol)) ++cnt;
    return cnt;
}

/*
 * Selected elements, each computed on its own from the definition:
 *   J[k][p][q] = sum_{r,s} kept (pq|rs) D_k[r][s]      (jidx holds p,q pairs)
 *   K[k][p][r] = sum_{q,s} kept (pq|rs) D_k[q][s]      (kidx holds p,r pairs)
 * Outputs are laid out [k][element].
 */
int oracle_jk_elements(int n, const double *center, const int32_t *nprim,
                       const double *exps, const double *w, const double *Q,
                       double tol, int m, const double *D,
                       int nj, const int32_t *jidx, double *Jout,
                       int nk, const int32_t *kidx, double *Kout)
{
    obasis b = mk_basis(n, center, nprim, exps, w);
    int64_t nn = (int64_t)n * n;
    for (int e = 0; e < nj; ++e) {
        int p = jidx[2 * e], q = jidx[2 * e + 1];
        for (int k = 0; k < m; ++k) Jout[(int64_t)k * nj + e] = 0.0;
        for (int r = 0; r < n; ++r)
            for (int s = 0; s < n; ++s) {
                if (!kept(Q, n, p, q, r, s, tol)) continue;
                double v = eri_c(&b, p, q, r, s);
                for (int k = 0; k < m; ++k)
                    Jout[(int64_t)k * nj + e] += D[k * nn + (int64_t)r * n + s] * v;
            }
    }
    for (int e = 0; e < nk; ++e) {
        int p = kidx[2 * e], r = kidx[2 * e + 1];
        for (int k = 0; k < m; ++k) Kout[(int64_t)k * nk + e] = 0.0;
        for (int q = 0; q < n; ++q)
            for (int s = 0; s < n; ++s) {
                if (!kept(Q, n, p, q, r, s, tol)) continue;
                double v = eri_c(&b, p, q, r, s);
                for (int k = 0; k < m; ++k)
                    Kout[(int64_t)k * nk + e] += D[k * nn + (int64_t)q * n + s] * v;
            }
    }
    free(b.off);
    return 0;
}

/*
 * Whole rows of J and K for selected row indices p (rows[i] = p):
 *   Jrow[k][i][q] = sum_{r,s} kept (pq|rs) D_k[r][s]
 *   Krow[k][i][r] = sum_{q,s} kept (pq|rs) D_k[q][s]
 * i.e. Eq. (J_and_K) for the elements J_pq and K_pr of row p, both sums
 * running over every integral (pq|rs) with first index p; each such integral
 * is evaluated once and used by both.  Outputs are laid out [k][i][column]
 * and overwritten.
 */
int oracle_jk_rows(int n, const double *center, const int32_t *nprim,
                   const double *exps, const double *w, const double *Q,
                   double tol, int m, const double *D,
                   int nrows, const int32_t *rows, double *Jrow, double *Krow)
{
    obasis b = mk_basis(n, center, nprim, exps, w);
    int64_t nn = (int64_t)n * n;
    double qmax = 0.0;
    for (int64_t e = 0; e < nn; ++e) if (Q[e] > qmax) qmax = Q[e];
    memset(Jrow, 0, sizeof(double) * (size_t)m * nrows * n);
    memset(Krow, 0, sizeof(double) * (size_t)m * nrows * n);
    for (int i = 0; i < nrows; ++i) {
        int p = rows[i];
        for (int q = 0; q < n; ++q) {
            /* no (pq|rs) can be kept when Q_pq times the largest Q is below tol */
            if (Q[(int64_t)p * n + q] * qmax < tol) continue;
            for (int r = 0; r < n; ++r)
                for (int s = 0; s < n; ++s) {
                    if (!kept(Q, n, p, q, r, s, tol)) continue;
                    double v = eri_c(&b, p, q, r, s);
                    for (int k = 0; k < m; ++k) {
                        const double *Dk = D + k * nn;
                        Jrow[((int64_t)k * nrows + i) * n + q] += Dk[(int64_t)r * n + s] * v;
                        Krow[((int64_t)k * nrows + i) * n + r] += Dk[(int64_t)q * n + s] * v;
                    }
                }
        }
    }
    free(b.off);
    return 0;
}

/*
 * Density fitting (the route the paper names as a future acceleration):
 * integrals with auxiliary s Gaussians chi_P(r) = exp(-c_P |r - C_P|^2)
 * (raw; the fitted J and K do not depend on how the auxiliaries are scaled).
 * Textbook closed forms, the ket of the four-centre formula reduced to one
 * Gaussian (q = c, Q = C, no ket prefactor):
 *   [ab|c] = 2 pi^{5/2} / (p c sqrt(p + c)) exp(-ab/p |AB|^2) F0(pc/(p+c) |PC|^2)
 *   [c|d]  = 2 pi^{5/2} / (c d sqrt(c + d)) F0(cd/(c+d) |CD|^2)
 * out3[(P n + p) n + q] = (pq|P) over the contracted orbitals; out2[P naux + Q] = (P|Q).
 */
static double prim_eri3(double a, const double *A, double b, const double *B,
                        double c, const double *C)
{
    double p = a + b, P[3], ab2 = 0, pc2 = 0;
    for (int x = 0; x < 3; ++x) {
        P[x] = (a * A[x] + b * B[x]) / p;
        ab2 += (A[x] - B[x]) * (A[x] - B[x]);
    }
    for (int x = 0; x < 3; ++x) pc2 += (P[x] - C[x]) * (P[x] - C[x]);
    return 2.0 * pow(OR_PI, 2.5) / (p * c * sqrt(p + c)) * exp(-a * b / p * ab2) *
           oracle_boys0(p * c / (p + c) * pc2);
}

int oracle_eri3(int n, const double *center, const int32_t *nprim, const double *exps,
                const double *w, int naux, const double *acenter, const double *aexp,
                double *out3)
{
    obasis b = mk_basis(n, center, nprim, exps, w);
    for (int P = 0; P < naux; ++P)
        for (int p = 0; p < n; ++p)
            for (int q = 0; q < n; ++q) {
                double v = 0.0;
                for (int64_t i = b.off[p]; i < b.off[p + 1]; ++i)
                    for (int64_t j = b.off[q]; j < b.off[q + 1]; ++j)
                        v += w[i] * w[j] * prim_eri3(exps[i], center + 3 * p, exps[j], center + 3 * q,
                                                     aexp[P], acenter + 3 * P);
                out3[((int64_t)P * n + p) * n + q] = v;
            }
    free(b.off);
    return 0;
}

int oracle_eri2(int naux, const double *acenter, const double *aexp, double *out2)
{
    for (int P = 0; P < naux; ++P)
        for (int Q = 0; Q < naux; ++Q) {
            double c = aexp[P], d = aexp[Q], r2 = 0.0;
            for (int x = 0; x < 3; ++x)
                r2 += (acenter[3 * P + x] - acenter[3 * Q + x]) * (acenter[3 * P + x] - acenter[3 * Q + x]);
            out2[(int64_t)P * naux + Q] = 2.0 * pow(OR_PI, 2.5) / (c * d * sqrt(c + d)) *
                                          oracle_boys0(c * d / (c + d) * r2);
        }
    return 0;
}

/*
 * Entry points for bases with Cartesian p and d functions (cart[i] in 0..9).
 * Normalisation (textbook Gaussian moments, int x^{2n} exp(-s x^2) dx =
 * (2n-1)!! / (2s)^n sqrt(pi/s)): a primitive with exponent triple (lx, ly, lz),
 * l = lx + ly + lz, has <g|g> = 1 for
 *   N = (2a/pi)^{3/4} (4a)^{l/2} / sqrt((2lx-1)!! (2ly-1)!! (2lz-1)!!),
 * and two primitives of one label on one centre overlap
 *   N_k N_j (pi/s)^{3/2} (2lx-1)!! (2ly-1)!! (2lz-1)!! / (2s)^l,  s = a_k + a_j.
 * w_k = c d_k N_k with c making the contracted function's norm one.
 */
static double dfact_odd(int l) /* (2l-1)!! for l = 0, 1, 2 */
{
    return l == 2 ? 3.0 : 1.0;
}

int oracle_normalize_l(int n, const int32_t *nprim, const double *exps,
                       const double *coefs, const int32_t *cart, double *w)
{
    if (n <= 0) return -1;
    int64_t *off = prim_offsets(n, nprim);
    for (int mu = 0; mu < n; ++mu) {
        int v[3];
        cart_vec(cart[mu], v);
        int l = v[0] + v[1] + v[2];
        double df = dfact_odd(v[0]) * dfact_odd(v[1]) * dfact_odd(v[2]);
        double s = 0.0;
        for (int64_t k = off[mu]; k < off[mu + 1]; ++k)
            for (int64_t j = off[mu]; j < off[mu + 1]; ++j) {
                double ak = exps[k], aj = exps[j], sk = ak + aj;
                double nk = pow(2.0 * ak / OR_PI, 0.75) * pow(4.0 * ak, 0.5 * l) / sqrt(df);
                double nj = pow(2.0 * aj / OR_PI, 0.75) * pow(4.0 * aj, 0.5 * l) / sqrt(df);
                double ov = pow(OR_PI / sk, 1.5) * df / pow(2.0 * sk, l);
                s += coefs[k] * coefs[j] * nk * nj * ov;
            }
        double c = 1.0 / sqrt(s);
        for (int64_t k = off[mu]; k < off[mu + 1]; ++k)
            w[k] = c * coefs[k] * pow(2.0 * exps[k] / OR_PI, 0.75) * pow(4.0 * exps[k], 0.5 * l) / sqrt(df);
    }
    free(off);
    return 0;
}

double oracle_eri_l(int n, const double *center, const int32_t *nprim, const double *exps,
                    const double *w, const int32_t *cart, int p, int q, int r, int s)
{
    obasis b = mk_basis(n, center, nprim, exps, w);
    b.cart = cart;
    double v = eri_c(&b, p, q, r, s);
    free(b.off);
    return v;
}

int oracle_eri_tensor_l(int n, const double *center, const int32_t *nprim, const double *exps,
                        const double *w, const int32_t *cart, double *out)
{
    obasis b = mk_basis(n, center, nprim, exps, w);
    b.cart = cart;
    for (int p = 0; p < n; ++p)
        for (int q = 0; q < n; ++q)
            for (int r = 0; r < n; ++r)
                for (int s = 0; s < n; ++s)
                    out[(((int64_t)p * n + q) * n + r) * n + s] = eri_c(&b, p, q, r, s);
    free(b.off);
    return 0;
}

int oracle_schwarz_l(int n, const double *center, const int32_t *nprim, const double *exps,
                     const double *w, const int32_t *cart, double *Q)
{
    obasis b = mk_basis(n, center, nprim, exps, w);
    b.cart = cart;
    for (int p = 0; p < n; ++p)
        for (int q = 0; q <= p; ++q) {
            double v = eri_c(&b, p, q, p, q);
            Q[(int64_t)p * n + q] = sqrt(v > 0.0 ? v : 0.0);
            Q[(int64_t)q * n + p] = Q[(int64_t)p * n + q];
        }
    free(b.off);
    return 0;
}

/* F_k = 2 J_k - K_k and t_k = D_k . F_k = sum_pq D_k[pq] F_k[pq] (Table I) */
int oracle_fock_traces(int n, int m, const double *D, const double *J,
                       const double *K, double *F, double *t)
{
    int64_t nn = (int64_t)n * n;
    for (int k = 0; k < m; ++k) {
        double acc = 0.0;
        for (int64_t e = 0; e < nn; ++e) {
            double f = 2.0 * J[k * nn + e] - K[k * nn + e];
            if (F) F[k * nn + e] = f;
            acc += D[k * nn + e] * f;
        }
        t[k] = acc;
    }
    return 0;
}
