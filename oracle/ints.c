/*
 * CPU oracle: one- and two-electron integrals over contracted Cartesian Gaussians, FP64.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, plain reference that the CUDA path is checked
 * against.  It shares no code, header, table or constant generator with the CUDA library, and the
 * product path never loads it.
 *
 * What it computes (all in bohr / hartree):
 *   - the integrals implied by the fragment Fock operator of the paper's Theory section,
 *     "Fragment Mean Field": h(1) (kinetic + nuclear attraction), the inter-fragment nuclear
 *     attraction h~ (the equation after Eq. wc), and the two-electron integrals (mu nu|lambda sigma)
 *     of Eq. dp2e;
 *   - by the Obara-Saika recurrences (Obara & Saika, J. Chem. Phys. 84, 3963 (1986)) for overlap,
 *     nuclear attraction and ERIs, written as plain recursions with memoisation and no HRR step;
 *   - kinetic energy from the second derivative of a 1D Cartesian Gaussian, expressed by overlaps;
 *   - the Boys function F_m(T) = int_0^1 t^(2m) exp(-T t^2) dt by its power series plus
 *     downward recursion (T < 30) and by erf plus upward recursion (T >= 30), using the C library's
 *     exp and erf.
 *
 * Basis convention: AO mu = ao_scale[mu] * sum_k coef[k] * x^lx y^ly z^lz exp(-alpha_k r^2), with
 * Cartesian components of a shell in lexicographic order (xx, xy, xz, yy, yz, zz).  ao_scale and
 * the coefficients are supplied by the caller.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define LMAX_CENTRE 2                 /* s, p, d */
#define NCART_ALL 10                  /* Cartesians with l <= 2 */
#define MMAX 16

typedef struct {
    int n_sh;
    const int* l;        /* [n_sh] */
    const int* np;       /* [n_sh] primitives */
    const int* p0;       /* [n_sh] offset into exp/coef */
    const int* ao0;      /* [n_sh] first AO of the shell */
    const double* xyz;   /* [n_sh*3] centre, bohr */
    const double* exps;
    const double* coef;
    const double* ao_scale; /* [n_ao] */
    int n_ao;
} or_shells;

static const double PI = 3.14159265358979323846;

/* ------------------------------------------------------------------------------- Boys function */

/* F_m(T) for m = 0..mmax (mmax <= MMAX). */
void or_boys(int mmax, double T, double* F)
{
    if (T < 30.0) {
        /* F_M(T) = exp(-T) * sum_k (2T)^k / ((2M+1)(2M+3)...(2M+2k+1)); all terms positive */
        int M = mmax;
        double term = 1.0 / (2.0 * M + 1.0), sum = term;
        for (int k = 1; k < 2000; ++k) {
            term *= 2.0 * T / (2.0 * M + 2.0 * k + 1.0);
            sum += term;
            if (term < 1e-18 * sum) break;
        }
        double e = exp(-T);
        F[M] = e * sum;
        /* downward: F_m = (2T F_{m+1} + exp(-T)) / (2m+1) */
        for (int m = M - 1; m >= 0; --m) F[m] = (2.0 * T * F[m + 1] + e) / (2.0 * m + 1.0);
    } else {
        double e = exp(-T);
        F[0] = 0.5 * sqrt(PI / T) * erf(sqrt(T));
        /* upward: F_{m+1} = ((2m+1) F_m - exp(-T)) / (2T) */
        for (int m = 0; m < mmax; ++m) F[m + 1] = ((2.0 * m + 1.0) * F[m] - e) / (2.0 * T);
    }
}

/* ------------------------------------------------------------------------------- Cartesian indexing */

static int ncart(int l) { return (l + 1) * (l + 2) / 2; }

/* k-th Cartesian of angular momentum l in lexicographic order */
static void cart_of(int l, int k, int c[3])
{
    int n = 0;
    for (int x = l; x >= 0; --x)
        for (int y = l - x; y >= 0; --y) {
            if (n == k) { c[0] = x; c[1] = y; c[2] = l - x - y; return; }
            ++n;
        }
}

/* index of (x,y,z) among all Cartesians with total l <= LMAX_CENTRE */
static int cart_index(const int c[3])
{
    int l = c[0] + c[1] + c[2];
    int base = l * (l + 1) * (l + 2) / 6;
    return base + (l - c[0]) * (l - c[0] + 1) / 2 + (l - c[0] - c[1]);
}

static double dist2(const double* A, const double* B)
{
    double dx = A[0] - B[0], dy = A[1] - B[1], dz = A[2] - B[2];
    return dx * dx + dy * dy + dz * dz;
}

/* ------------------------------------------------------------------------------- overlap / kinetic */

/* 1D overlap S_ij of x^i exp(-a x^2) (centre A) and x^j exp(-b x^2) (centre B), Obara-Saika:
 * S_{i+1,j} = X_PA S_ij + (i S_{i-1,j} + j S_{i,j-1}) / (2p),
 * S_{i,j+1} = X_PB S_ij + (i S_{i-1,j} + j S_{i,j-1}) / (2p),
 * S_00 = sqrt(pi/p) exp(-ab/p X_AB^2). */
static void overlap_1d(int imax, int jmax, double a, double b, double A, double B, double S[8][8])
{
    double p = a + b, P = (a * A + b * B) / p;
    double XPA = P - A, XPB = P - B;
    S[0][0] = sqrt(PI / p) * exp(-a * b / p * (A - B) * (A - B));
    for (int i = 0; i <= imax; ++i)
        for (int j = 0; j <= jmax; ++j) {
            if (i == 0 && j == 0) continue;
            double v;
            if (i > 0) {
                v = XPA * S[i - 1][j];
                if (i > 1) v += (i - 1) * S[i - 2][j] / (2 * p);
                if (j > 0) v += j * S[i - 1][j - 1] / (2 * p);
            } else {
                v = XPB * S[i][j - 1];
                if (j > 1) v += (j - 1) * S[i][j - 2] / (2 * p);
            }
            S[i][j] = v;
        }
}

/* S (and optionally T) for one shell set; out[mu*n_ao+nu] */
static void one_electron_st(const or_shells* s, double* Sout, double* Tout)
{
    int n = s->n_ao;
    if (Sout) memset(Sout, 0, sizeof(double) * n * n);
    if (Tout) memset(Tout, 0, sizeof(double) * n * n);
    for (int sa = 0; sa < s->n_sh; ++sa)
        for (int sb = 0; sb < s->n_sh; ++sb) {
            int la = s->l[sa], lb = s->l[sb];
            const double* A = s->xyz + 3 * sa;
            const double* B = s->xyz + 3 * sb;
            for (int ka = 0; ka < s->np[sa]; ++ka)
                for (int kb = 0; kb < s->np[sb]; ++kb) {
                    double a = s->exps[s->p0[sa] + ka], b = s->exps[s->p0[sb] + kb];
                    double cc = s->coef[s->p0[sa] + ka] * s->coef[s->p0[sb] + kb];
                    double S1[3][8][8];
                    for (int d = 0; d < 3; ++d) overlap_1d(la, lb + 2, a, b, A[d], B[d], S1[d]);
                    for (int ia = 0; ia < ncart(la); ++ia)
                        for (int ib = 0; ib < ncart(lb); ++ib) {
                            int ca[3], cb[3];
                            cart_of(la, ia, ca);
                            cart_of(lb, ib, cb);
                            double s3 = S1[0][ca[0]][cb[0]] * S1[1][ca[1]][cb[1]] * S1[2][ca[2]][cb[2]];
                            int mu = s->ao0[sa] + ia, nu = s->ao0[sb] + ib;
                            double sc = cc * s->ao_scale[mu] * s->ao_scale[nu];
                            if (Sout) Sout[mu * n + nu] += sc * s3;
                            if (Tout) {
                                /* d^2/dx^2 [x^j e^{-b x^2}] = j(j-1) x^{j-2} - 2b(2j+1) x^j + 4b^2 x^{j+2} */
                                double D1[3];
                                for (int d = 0; d < 3; ++d) {
                                    int i = ca[d], j = cb[d];
                                    double v = -2.0 * b * (2 * j + 1) * S1[d][i][j] + 4.0 * b * b * S1[d][i][j + 2];
                                    if (j >= 2) v += j * (j - 1) * S1[d][i][j - 2];
                                    D1[d] = v;
                                }
                                double t = D1[0] * S1[1][ca[1]][cb[1]] * S1[2][ca[2]][cb[2]]
                                         + S1[0][ca[0]][cb[0]] * D1[1] * S1[2][ca[2]][cb[2]]
                                         + S1[0][ca[0]][cb[0]] * S1[1][ca[1]][cb[1]] * D1[2];
                                Tout[mu * n + nu] += sc * (-0.5) * t;
                            }
                        }
                }
        }
}

/* Cartesian moment integrals about the point c: out[k][mu][nu] = <mu| (r - c)^k |nu> for k = 1, x, y, z,
 * xx, xy, xz, yy, yz, zz.  In 1D, (x - c) x_B^j = x_B^{j+1} + (B - c) x_B^j, so every moment is a
 * combination of overlaps with the ket's power raised by up to 2. */
void or_moments(const or_shells* s, const double* c, double* out)
{
    int n = s->n_ao;
    memset(out, 0, sizeof(double) * 10 * n * n);
    for (int sa = 0; sa < s->n_sh; ++sa)
        for (int sb = 0; sb < s->n_sh; ++sb) {
            int la = s->l[sa], lb = s->l[sb];
            const double* A = s->xyz + 3 * sa;
            const double* B = s->xyz + 3 * sb;
            for (int ka = 0; ka < s->np[sa]; ++ka)
                for (int kb = 0; kb < s->np[sb]; ++kb) {
                    double a = s->exps[s->p0[sa] + ka], b = s->exps[s->p0[sb] + kb];
                    double cc = s->coef[s->p0[sa] + ka] * s->coef[s->p0[sb] + kb];
                    double S1[3][8][8];
                    for (int d = 0; d < 3; ++d) overlap_1d(la, lb + 2, a, b, A[d], B[d], S1[d]);
                    for (int ia = 0; ia < ncart(la); ++ia)
                        for (int ib = 0; ib < ncart(lb); ++ib) {
                            int ca[3], cb[3];
                            cart_of(la, ia, ca);
                            cart_of(lb, ib, cb);
                            double m[3][3]; /* m[d][k]: 1D moment of order k in direction d */
                            for (int d = 0; d < 3; ++d) {
                                int i = ca[d], j = cb[d];
                                double bc = B[d] - c[d];
                                m[d][0] = S1[d][i][j];
                                m[d][1] = S1[d][i][j + 1] + bc * S1[d][i][j];
                                m[d][2] = S1[d][i][j + 2] + 2.0 * bc * S1[d][i][j + 1] + bc * bc * S1[d][i][j];
                            }
                            const int kk[10][3] = {{0, 0, 0}, {1, 0, 0}, {0, 1, 0}, {0, 0, 1}, {2, 0, 0},
                                                   {1, 1, 0}, {1, 0, 1}, {0, 2, 0}, {0, 1, 1}, {0, 0, 2}};
                            int mu = s->ao0[sa] + ia, nu = s->ao0[sb] + ib;
                            double sc = cc * s->ao_scale[mu] * s->ao_scale[nu];
                            for (int k = 0; k < 10; ++k)
                                out[(size_t)k * n * n + mu * n + nu] +=
                                    sc * m[0][kk[k][0]] * m[1][kk[k][1]] * m[2][kk[k][2]];
                        }
                }
        }
}

void or_overlap(const or_shells* s, double* S) { one_electron_st(s, S, NULL); }
void or_kinetic(const or_shells* s, double* T) { one_electron_st(s, NULL, T); }

/* ------------------------------------------------------------------------------- nuclear attraction */

typedef struct {
    double PA[3], PB[3], PC[3], p;
    double base[MMAX + 1];
    double memo[NCART_ALL][NCART_ALL][MMAX + 1];
    int stamp[NCART_ALL][NCART_ALL][MMAX + 1];
    int gen;
} nuc_ctx;

/* [a|C|b]^(m), Obara-Saika:
 * [a+1_i|b]^(m) = PA_i [a|b]^(m) - PC_i [a|b]^(m+1)
 *               + a_i/(2p) ([a-1_i|b]^(m) - [a-1_i|b]^(m+1)) + b_i/(2p) ([a|b-1_i]^(m) - [a|b-1_i]^(m+1))
 * and the same with PB for b; [0|0]^(m) = (2 pi/p) K_ab F_m(p PC^2). */
static double nuc_r(nuc_ctx* c, const int a[3], const int b[3], int m)
{
    int La = a[0] + a[1] + a[2], Lb = b[0] + b[1] + b[2];
    if (La == 0 && Lb == 0) return c->base[m];
    int ia = cart_index(a), ib = cart_index(b);
    if (c->stamp[ia][ib][m] == c->gen) return c->memo[ia][ib][m];
    int A[3] = {a[0], a[1], a[2]}, B[3] = {b[0], b[1], b[2]};
    double v;
    int i;
    if (La > 0) {
        i = a[0] ? 0 : (a[1] ? 1 : 2);
        A[i] -= 1;
        v = c->PA[i] * nuc_r(c, A, B, m) - c->PC[i] * nuc_r(c, A, B, m + 1);
        if (A[i] > 0) {
            int A2[3] = {A[0], A[1], A[2]};
            A2[i] -= 1;
            v += A[i] / (2 * c->p) * (nuc_r(c, A2, B, m) - nuc_r(c, A2, B, m + 1));
        }
        if (B[i] > 0) {
            int B2[3] = {B[0], B[1], B[2]};
            B2[i] -= 1;
            v += B[i] / (2 * c->p) * (nuc_r(c, A, B2, m) - nuc_r(c, A, B2, m + 1));
        }
    } else {
        i = b[0] ? 0 : (b[1] ? 1 : 2);
        B[i] -= 1;
        v = c->PB[i] * nuc_r(c, A, B, m) - c->PC[i] * nuc_r(c, A, B, m + 1);
        if (B[i] > 0) {
            int B2[3] = {B[0], B[1], B[2]};
            B2[i] -= 1;
            v += B[i] / (2 * c->p) * (nuc_r(c, A, B2, m) - nuc_r(c, A, B2, m + 1));
        }
    }
    c->stamp[ia][ib][m] = c->gen;
    c->memo[ia][ib][m] = v;
    return v;
}

/* V_mu nu = - sum_C Z_C <mu| 1/|r - R_C| |nu> */
void or_nuclear(const or_shells* s, int n_c, const double* c_xyz, const double* c_Z, double* V)
{
    int n = s->n_ao;
    memset(V, 0, sizeof(double) * n * n);
    nuc_ctx* c = (nuc_ctx*)calloc(1, sizeof(nuc_ctx));
    for (int sa = 0; sa < s->n_sh; ++sa)
        for (int sb = 0; sb < s->n_sh; ++sb) {
            int la = s->l[sa], lb = s->l[sb];
            const double* A = s->xyz + 3 * sa;
            const double* B = s->xyz + 3 * sb;
            for (int ka = 0; ka < s->np[sa]; ++ka)
                for (int kb = 0; kb < s->np[sb]; ++kb) {
                    double a = s->exps[s->p0[sa] + ka], b = s->exps[s->p0[sb] + kb];
                    double cc = s->coef[s->p0[sa] + ka] * s->coef[s->p0[sb] + kb];
                    double p = a + b, P[3];
                    for (int d = 0; d < 3; ++d) P[d] = (a * A[d] + b * B[d]) / p;
                    double Kab = exp(-a * b / p * dist2(A, B));
                    for (int ic = 0; ic < n_c; ++ic) {
                        const double* C = c_xyz + 3 * ic;
                        c->p = p;
                        for (int d = 0; d < 3; ++d) {
                            c->PA[d] = P[d] - A[d];
                            c->PB[d] = P[d] - B[d];
                            c->PC[d] = P[d] - C[d];
                        }
                        double F[MMAX + 1];
                        or_boys(la + lb, p * dist2(P, C), F);
                        for (int m = 0; m <= la + lb; ++m) c->base[m] = 2 * PI / p * Kab * F[m];
                        c->gen++;
                        for (int ia = 0; ia < ncart(la); ++ia)
                            for (int ib = 0; ib < ncart(lb); ++ib) {
                                int ca[3], cb[3];
                                cart_of(la, ia, ca);
                                cart_of(lb, ib, cb);
                                int mu = s->ao0[sa] + ia, nu = s->ao0[sb] + ib;
                                V[mu * n + nu] -= c_Z[ic] * cc * s->ao_scale[mu] * s->ao_scale[nu] * nuc_r(c, ca, cb, 0);
                            }
                    }
                }
        }
    free(c);
}

/* ------------------------------------------------------------------------------- ERIs */

typedef struct {
    double PA[3], PB[3], QC[3], QD[3], WP[3], WQ[3];
    double zeta, eta, rho;
    double base[MMAX + 1];
    double memo[NCART_ALL][NCART_ALL][NCART_ALL][NCART_ALL][MMAX + 1];
    int stamp[NCART_ALL][NCART_ALL][NCART_ALL][NCART_ALL][MMAX + 1];
    int gen;
} eri_ctx;

static int Lsum(const int a[3]) { return a[0] + a[1] + a[2]; }

/* [ab|cd]^(m) by the Obara-Saika recurrence (transfer to the first centre with non-zero l):
 * [a+1_i,b|cd]^(m) = PA_i [ab|cd]^(m) + WP_i [ab|cd]^(m+1)
 *   + a_i/(2 zeta) ([a-1_i,b|cd]^(m) - rho/zeta [a-1_i,b|cd]^(m+1))
 *   + b_i/(2 zeta) ([a,b-1_i|cd]^(m) - rho/zeta [a,b-1_i|cd]^(m+1))
 *   + c_i/(2(zeta+eta)) [ab|c-1_i,d]^(m+1) + d_i/(2(zeta+eta)) [ab|c,d-1_i]^(m+1),
 * the same with PB for b, and the ket analogues with QC/QD, WQ, eta.
 * [00|00]^(m) = 2 pi^(5/2) / (zeta eta sqrt(zeta+eta)) K_ab K_cd F_m(rho |PQ|^2). */
static double eri_r(eri_ctx* c, const int a[3], const int b[3], const int cc_[3], const int d[3], int m)
{
    int La = Lsum(a), Lb = Lsum(b), Lc = Lsum(cc_), Ld = Lsum(d);
    if (La + Lb + Lc + Ld == 0) return c->base[m];
    int ia = cart_index(a), ib = cart_index(b), ic = cart_index(cc_), id = cart_index(d);
    if (c->stamp[ia][ib][ic][id][m] == c->gen) return c->memo[ia][ib][ic][id][m];
    int A[3] = {a[0], a[1], a[2]}, B[3] = {b[0], b[1], b[2]};
    int C[3] = {cc_[0], cc_[1], cc_[2]}, D[3] = {d[0], d[1], d[2]};
    double z = c->zeta, e = c->eta, r = c->rho, v = 0.0;
    int i;
    int *X, *Y, *U, *W; /* X: centre reduced; Y: its partner; U, W: the other side */
    const double *XA, *WX;
    double ex;       /* exponent of the side of X */
    if (La > 0)      { X = A; Y = B; U = C; W = D; XA = c->PA; WX = c->WP; ex = z; }
    else if (Lb > 0) { X = B; Y = A; U = C; W = D; XA = c->PB; WX = c->WP; ex = z; }
    else if (Lc > 0) { X = C; Y = D; U = A; W = B; XA = c->QC; WX = c->WQ; ex = e; }
    else             { X = D; Y = C; U = A; W = B; XA = c->QD; WX = c->WQ; ex = e; }
    i = X[0] ? 0 : (X[1] ? 1 : 2);
    X[i] -= 1;
    v = XA[i] * eri_r(c, A, B, C, D, m) + WX[i] * eri_r(c, A, B, C, D, m + 1);
    if (X[i] > 0) {
        X[i] -= 1;
        v += (X[i] + 1) / (2 * ex) * (eri_r(c, A, B, C, D, m) - r / ex * eri_r(c, A, B, C, D, m + 1));
        X[i] += 1;
    }
    if (Y[i] > 0) {
        int n = Y[i];
        Y[i] -= 1;
        v += n / (2 * ex) * (eri_r(c, A, B, C, D, m) - r / ex * eri_r(c, A, B, C, D, m + 1));
        Y[i] += 1;
    }
    if (U[i] > 0) {
        int n = U[i];
        U[i] -= 1;
        v += n / (2 * (z + e)) * eri_r(c, A, B, C, D, m + 1);
        U[i] += 1;
    }
    if (W[i] > 0) {
        int n = W[i];
        W[i] -= 1;
        v += n / (2 * (z + e)) * eri_r(c, A, B, C, D, m + 1);
        W[i] += 1;
    }
    c->stamp[ia][ib][ic][id][m] = c->gen;
    c->memo[ia][ib][ic][id][m] = v;
    return v;
}

/* Contracted shell quartet (ab|cd) -> out[((ia*nb + ib)*nc + ic)*nd + id], normalised AOs. */
static void eri_shell_quartet(eri_ctx* c, const or_shells* s1, int sa, int sb, const or_shells* s2, int sc,
                              int sd, double* out)
{
    int la = s1->l[sa], lb = s1->l[sb], lc = s2->l[sc], ld = s2->l[sd];
    int na = ncart(la), nb = ncart(lb), nc = ncart(lc), nd = ncart(ld);
    int ntot = na * nb * nc * nd;
    for (int k = 0; k < ntot; ++k) out[k] = 0.0;
    const double *A = s1->xyz + 3 * sa, *B = s1->xyz + 3 * sb, *C = s2->xyz + 3 * sc, *D = s2->xyz + 3 * sd;
    int L = la + lb + lc + ld;
    for (int ka = 0; ka < s1->np[sa]; ++ka)
        for (int kb = 0; kb < s1->np[sb]; ++kb) {
            double a = s1->exps[s1->p0[sa] + ka], b = s1->exps[s1->p0[sb] + kb];
            double cab = s1->coef[s1->p0[sa] + ka] * s1->coef[s1->p0[sb] + kb];
            double z = a + b, P[3];
            for (int d = 0; d < 3; ++d) P[d] = (a * A[d] + b * B[d]) / z;
            double Kab = exp(-a * b / z * dist2(A, B));
            for (int kc = 0; kc < s2->np[sc]; ++kc)
                for (int kd = 0; kd < s2->np[sd]; ++kd) {
                    double g = s2->exps[s2->p0[sc] + kc], h = s2->exps[s2->p0[sd] + kd];
                    double ccd = s2->coef[s2->p0[sc] + kc] * s2->coef[s2->p0[sd] + kd];
                    double e = g + h, Q[3], W[3];
                    for (int d = 0; d < 3; ++d) Q[d] = (g * C[d] + h * D[d]) / e;
                    double Kcd = exp(-g * h / e * dist2(C, D));
                    double rho = z * e / (z + e);
                    for (int d = 0; d < 3; ++d) {
                        W[d] = (z * P[d] + e * Q[d]) / (z + e);
                        c->PA[d] = P[d] - A[d];
                        c->PB[d] = P[d] - B[d];
                        c->QC[d] = Q[d] - C[d];
                        c->QD[d] = Q[d] - D[d];
                        c->WP[d] = W[d] - P[d];
                        c->WQ[d] = W[d] - Q[d];
                    }
                    c->zeta = z;
                    c->eta = e;
                    c->rho = rho;
                    double F[MMAX + 1];
                    or_boys(L, rho * dist2(P, Q), F);
                    double pre = 2.0 * pow(PI, 2.5) / (z * e * sqrt(z + e)) * Kab * Kcd;
                    for (int m = 0; m <= L; ++m) c->base[m] = pre * F[m];
                    c->gen++;
                    double cc4 = cab * ccd;
                    int k = 0;
                    for (int ia = 0; ia < na; ++ia) {
                        int ca[3];
                        cart_of(la, ia, ca);
                        for (int ib = 0; ib < nb; ++ib) {
                            int cb[3];
                            cart_of(lb, ib, cb);
                            for (int ic = 0; ic < nc; ++ic) {
                                int cc[3];
                                cart_of(lc, ic, cc);
                                for (int id = 0; id < nd; ++id, ++k) {
                                    int cd[3];
                                    cart_of(ld, id, cd);
                                    out[k] += cc4 * eri_r(c, ca, cb, cc, cd, 0);
                                }
                            }
                        }
                    }
                }
        }
    int k = 0;
    for (int ia = 0; ia < na; ++ia)
        for (int ib = 0; ib < nb; ++ib)
            for (int ic = 0; ic < nc; ++ic)
                for (int id = 0; id < nd; ++id, ++k)
                    out[k] *= s1->ao_scale[s1->ao0[sa] + ia] * s1->ao_scale[s1->ao0[sb] + ib] *
                              s2->ao_scale[s2->ao0[sc] + ic] * s2->ao_scale[s2->ao0[sd] + id];
}

/* Schwarz factors Q[a*n_sh+b] = max_{mu in a, nu in b} sqrt|(mu nu|mu nu)| */
void or_schwarz(const or_shells* s, double* Q)
{
    int n = s->n_sh;
#pragma omp parallel
    {
        eri_ctx* c = (eri_ctx*)calloc(1, sizeof(eri_ctx));
        double buf[6 * 6 * 6 * 6];
#pragma omp for schedule(dynamic)
        for (int ab = 0; ab < n * n; ++ab) {
            int sa = ab / n, sb = ab % n;
            eri_shell_quartet(c, s, sa, sb, s, sa, sb, buf);
            int na = ncart(s->l[sa]), nb = ncart(s->l[sb]);
            double q = 0.0;
            for (int ia = 0; ia < na; ++ia)
                for (int ib = 0; ib < nb; ++ib) {
                    double v = fabs(buf[((ia * nb + ib) * na + ia) * nb + ib]);
                    if (v > q) q = v;
                }
            Q[ab] = sqrt(q);
        }
        free(c);
    }
}

/* ERI block (mu nu|lambda sigma) with mu,nu in s1 and lambda,sigma in s2:
 * out[((mu*n1 + nu)*n2 + lambda)*n2 + sigma].  If Q1/Q2 are given, a shell quartet with
 * Q1[ab]*Q2[cd] < tau is set to zero (Schwarz screening). */
void or_eri_block(const or_shells* s1, const or_shells* s2, const double* Q1, const double* Q2, double tau,
                  double* out)
{
    int n1 = s1->n_ao, n2 = s2->n_ao;
    int nsh1 = s1->n_sh, nsh2 = s2->n_sh;
    memset(out, 0, sizeof(double) * (size_t)n1 * n1 * n2 * n2);
#pragma omp parallel
    {
        eri_ctx* c = (eri_ctx*)calloc(1, sizeof(eri_ctx));
        double buf[6 * 6 * 6 * 6];
#pragma omp for schedule(dynamic)
        for (int ab = 0; ab < nsh1 * nsh1; ++ab) {
            int sa = ab / nsh1, sb = ab % nsh1;
            for (int sc = 0; sc < nsh2; ++sc)
                for (int sd = 0; sd < nsh2; ++sd) {
                    if (Q1 && Q2 && Q1[ab] * Q2[sc * nsh2 + sd] < tau) continue;
                    eri_shell_quartet(c, s1, sa, sb, s2, sc, sd, buf);
                    int na = ncart(s1->l[sa]), nb = ncart(s1->l[sb]), nc = ncart(s2->l[sc]), nd = ncart(s2->l[sd]);
                    int k = 0;
                    for (int ia = 0; ia < na; ++ia)
                        for (int ib = 0; ib < nb; ++ib)
                            for (int ic = 0; ic < nc; ++ic)
                                for (int id = 0; id < nd; ++id, ++k) {
                                    size_t mu = s1->ao0[sa] + ia, nu = s1->ao0[sb] + ib;
                                    size_t la = s2->ao0[sc] + ic, si = s2->ao0[sd] + id;
                                    out[((mu * n1 + nu) * n2 + la) * n2 + si] = buf[k];
                                }
                }
        }
        free(c);
    }
}

/* Number of shell quartets (ab|cd), a<=b in s1, c<=d in s2, that survive Q1[ab]Q2[cd] >= tau. */
long long or_count_quartets(const or_shells* s1, const or_shells* s2, const double* Q1, const double* Q2,
                            double tau)
{
    long long n = 0;
    for (int sa = 0; sa < s1->n_sh; ++sa)
        for (int sb = sa; sb < s1->n_sh; ++sb)
            for (int sc = 0; sc < s2->n_sh; ++sc)
                for (int sd = sc; sd < s2->n_sh; ++sd)
                    if (Q1[sa * s1->n_sh + sb] * Q2[sc * s2->n_sh + sd] >= tau) ++n;
    return n;
}
