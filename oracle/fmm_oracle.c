/*
 * fmm_oracle.c -- plain, serial, FP64 CPU oracle for the fast multipole method of
 * Dehnen, "A fast multipole method for stellar dynamics" (arXiv 1405.2255).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, literal restatement of the
 * paper's method that the GPU library is checked against.  Only the test suite,
 * the smoke check and the CPU-baseline leg of the benchmark load it.  It shares no
 * code, header, table or constant with the CUDA library, and it never calls it.
 *
 * What it follows (section / equation of the paper):
 *   - direct summation, eq. (1) for Psi and a, eq. (6) for the scale f;
 *   - solid harmonics Theta_n^m, Upsilon_n^m, eq. (2), evaluated with the
 *     recurrences of App. A.3.1 (Theta_n^n, Upsilon_n^n and the three-term
 *     recurrences in n), negative m from the symmetry X_n^{-m} = (-1)^m X_n^{m*};
 *   - P2M eq. (3c), M2M eq. (4), M2L eq. (3b), L2L eq. (5), L2P eq. (7);
 *   - the swap matrices of App. A.5.1 (recurrences) and the rotation-accelerated M2L of
 *     App. A.5.2 with the z-axis kernel eq. (A31) (used by the tests only; the oracle's
 *     FMM takes eq. (3b) term by term);
 *     a = -(Re Psi_1^1, Im Psi_1^1, Psi_1^0) (Sec. 2.1);
 *   - oct-tree of cubic cells (Sec. 2.2), expansion centres z = s = centre of the
 *     smallest enclosing sphere (Sec. 5.1.1), radii rho (Sec. 4, eqs. 9-10);
 *   - multipole power P_n eq. (14), E_{A->B} eq. (15), E~ eq. (17);
 *   - the one-sided dual tree walk (Sec. 2.2.2, Sec. 6.1) with the error-balanced
 *     acceptance criteria eqs. (18a,b) or the geometric one eq. (9);
 *   - the low-order FMM estimate of a_b (p=1) or f_b (p=0) with theta<1 and
 *     z = s = centre of mass (Sec. 5.3.2).
 *
 * Readings where the paper is silent (each one is listed in the design notes):
 *   R-box   root cube side = max extent * (1 + 2^-20), anchored at the lower corner.
 *   R-key   63-bit Morton key, 21 bits per axis, x in the most significant bit of
 *           each triplet; sort by (key, original index).
 *   R-leaf  a cell is split iff it holds more than leaf_size particles and is above
 *           depth 21; daughters are the non-empty octants in key order.
 *   R-ses   leaf centre: smallest enclosing ball of its particles (Welzl, the
 *           first 128 particles taken in bit-reversed index order; with the
 *           move-to-front rule for leaves of at most 128 particles);
 *           internal centre: smallest ball enclosing the daughters' balls
 *           (s_d, rho_d) (enumeration of support sets of up to 4 balls); both in
 *           IEEE single precision relative to the cell's first particle / first
 *           daughter centre; rho = exact FP64 max over the particles of |x - s|.
 *   R-p2p   a pair (A,B) is summed directly when N_A*N_B < p2p_c * p^3 (checked
 *           first: the descendants of such a pair would all be summed directly),
 *           p being the order of the expansion in use (1 or 0 in the estimate).
 *   R-split split the cell with the larger rho (ties: A); never a leaf; A = B
 *           splits into all ordered daughter pairs.
 *   R-mac   (18a,b) as strict inequalities; E~ M_A/r^2 is evaluated without
 *           dividing by M_A; the factor 8 max/(rhoA+rhoB) is 8 when both radii are 0.
 *   R-coin  pairs at distance 0 contribute nothing and are counted.
 *   R-G     everything is computed with G = 1 and Psi, a are multiplied by G last.
 *
 * Precision: IEEE FP64 throughout; build with -ffp-contract=off.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cplx;

/* index of (n, m), -n <= m <= n, in a full complex harmonic array of (p+1)^2 */
static inline int IX(int n, int m) { return n * n + n + m; }
static inline int NCOEF(int p) { return (p + 1) * (p + 1); }
static inline double sgn_m(int m) { return (m & 1) ? -1.0 : 1.0; }

/* ------------------------------------------------------------------------- */
/* Solid harmonics (eq. 2; recurrences App. A.3.1)                            */
/* ------------------------------------------------------------------------- */

/* Upsilon_n^m(r): Upsilon_0^0 = 1, Upsilon_n^n = (x+iy)/(2n) Upsilon_{n-1}^{n-1},
 * (n^2-m^2) Upsilon_n^m = (2n-1) z Upsilon_{n-1}^m - r^2 Upsilon_{n-2}^m. */
void orc_upsilon(int p, double x, double y, double z, cplx *Y)
{
    const double r2 = x * x + y * y + z * z;
    const cplx xi = x + I * y;
    Y[IX(0, 0)] = 1.0;
    for (int m = 0; m <= p; ++m) {
        if (m > 0) Y[IX(m, m)] = xi / (2.0 * m) * Y[IX(m - 1, m - 1)];
        for (int n = m + 1; n <= p; ++n) {
            cplx two_back = (n - 2 >= m) ? Y[IX(n - 2, m)] : 0.0;
            Y[IX(n, m)] = ((2.0 * n - 1.0) * z * Y[IX(n - 1, m)] - r2 * two_back) /
                          (double)(n * n - m * m);
        }
    }
    for (int n = 1; n <= p; ++n)
        for (int m = 1; m <= n; ++m) Y[IX(n, -m)] = sgn_m(m) * conj(Y[IX(n, m)]);
}

/* Theta_n^m(r): Theta_0^0 = 1/r, Theta_n^n = (2n-1)(x+iy)/r^2 Theta_{n-1}^{n-1},
 * r^2 Theta_n^m = (2n-1) z Theta_{n-1}^m - ((n-1)^2 - m^2) Theta_{n-2}^m. */
void orc_theta(int p, double x, double y, double z, cplx *T)
{
    const double r2 = x * x + y * y + z * z;
    const cplx xi = x + I * y;
    T[IX(0, 0)] = 1.0 / sqrt(r2);
    for (int m = 0; m <= p; ++m) {
        if (m > 0) T[IX(m, m)] = (2.0 * m - 1.0) * xi / r2 * T[IX(m - 1, m - 1)];
        for (int n = m + 1; n <= p; ++n) {
            cplx two_back = (n - 2 >= m) ? T[IX(n - 2, m)] : 0.0;
            double c2 = (double)((n - 1) * (n - 1) - m * m);
            T[IX(n, m)] = ((2.0 * n - 1.0) * z * T[IX(n - 1, m)] - c2 * two_back) / r2;
        }
    }
    for (int n = 1; n <= p; ++n)
        for (int m = 1; m <= n; ++m) T[IX(n, -m)] = sgn_m(m) * conj(T[IX(n, m)]);
}

/* real views used by the tests: U_n^m, T_n^m of eqs. (A24) */
void orc_upsilon_re(int p, double x, double y, double z, double *re, double *im)
{
    cplx *Y = malloc(sizeof(cplx) * NCOEF(p));
    orc_upsilon(p, x, y, z, Y);
    for (int i = 0; i < NCOEF(p); ++i) { re[i] = creal(Y[i]); im[i] = cimag(Y[i]); }
    free(Y);
}
void orc_theta_re(int p, double x, double y, double z, double *re, double *im)
{
    cplx *T = malloc(sizeof(cplx) * NCOEF(p));
    orc_theta(p, x, y, z, T);
    for (int i = 0; i < NCOEF(p); ++i) { re[i] = creal(T[i]); im[i] = cimag(T[i]); }
    free(T);
}

/* ------------------------------------------------------------------------- */
/* FMM kernels, literally eqs. (3a-c), (4), (5), (7)                          */
/* ------------------------------------------------------------------------- */

/* eq. (3c): M_n^m(z) += sum_a mu_a Upsilon_n^m(x_a - z) */
static void p2m(int p, long n, const double *x, const double *mu, const double z[3], cplx *M)
{
    cplx *Y = malloc(sizeof(cplx) * NCOEF(p));
    for (long a = 0; a < n; ++a) {
        orc_upsilon(p, x[3 * a] - z[0], x[3 * a + 1] - z[1], x[3 * a + 2] - z[2], Y);
        for (int i = 0; i < NCOEF(p); ++i) M[i] += mu[a] * Y[i];
    }
    free(Y);
}

/* eq. (4): Mout_n^m(z') += sum_{k<=n} sum_l Upsilon_k^l(z - z') M_{n-k}^{m-l}(z) */
static void m2m(int p, const cplx *M, const double z[3], const double zp[3], cplx *Mout)
{
    cplx *Y = malloc(sizeof(cplx) * NCOEF(p));
    orc_upsilon(p, z[0] - zp[0], z[1] - zp[1], z[2] - zp[2], Y);
    for (int n = 0; n <= p; ++n)
        for (int m = -n; m <= n; ++m) {
            cplx s = 0;
            for (int k = 0; k <= n; ++k)
                for (int l = -k; l <= k; ++l) {
                    int nn = n - k, mm = m - l;
                    if (mm < -nn || mm > nn) continue;
                    s += Y[IX(k, l)] * M[IX(nn, mm)];
                }
            Mout[IX(n, m)] += s;
        }
    free(Y);
}

/* eq. (3b): F_n^m(s_B) += sum_{k<=p-n} sum_l M_k^{l*}(z_A) Theta_{n+k}^{m+l}(s_B - z_A) */
static void m2l(int p, const cplx *M, const double zA[3], const double sB[3], cplx *F)
{
    cplx *T = malloc(sizeof(cplx) * NCOEF(p));
    orc_theta(p, sB[0] - zA[0], sB[1] - zA[1], sB[2] - zA[2], T);
    for (int n = 0; n <= p; ++n)
        for (int m = -n; m <= n; ++m) {
            cplx s = 0;
            for (int k = 0; k <= p - n; ++k)
                for (int l = -k; l <= k; ++l) {
                    int nn = n + k, mm = m + l;
                    if (mm < -nn || mm > nn) continue;
                    s += conj(M[IX(k, l)]) * T[IX(nn, mm)];
                }
            F[IX(n, m)] += s;
        }
    free(T);
}

/* eq. (5): Fout_n^m(s') += sum_{k<=p-n} sum_l Upsilon_k^{l*}(s - s') F_{n+k}^{m+l}(s) */
static void l2l(int p, const cplx *F, const double s[3], const double sp[3], cplx *Fout)
{
    cplx *Y = malloc(sizeof(cplx) * NCOEF(p));
    orc_upsilon(p, s[0] - sp[0], s[1] - sp[1], s[2] - sp[2], Y);
    for (int n = 0; n <= p; ++n)
        for (int m = -n; m <= n; ++m) {
            cplx acc = 0;
            for (int k = 0; k <= p - n; ++k)
                for (int l = -k; l <= k; ++l) {
                    int nn = n + k, mm = m + l;
                    if (mm < -nn || mm > nn) continue;
                    acc += conj(Y[IX(k, l)]) * F[IX(nn, mm)];
                }
            Fout[IX(n, m)] += acc;
        }
    free(Y);
}

/* eqs. (3a), (7): Psi_n^m(x_b) = sum_{k<=p-n} sum_l Upsilon_k^{l*}(s_B - x_b) F_{n+k}^{m+l}(s_B),
 * returns Psi = Psi_0^0 and a = -(Re Psi_1^1, Im Psi_1^1, Psi_1^0). */
/* tidal tensor of Sec. 7.4 from Psi_2^m: T = (xx, xy, xz, yy, yz, zz).  Reading R-tidal:
 * the paper prints T_xy = -Im{Psi_2^2}/2; with the harmonics of App. A.3 (the same that give
 * a = -(Re Psi_1^1, Im Psi_1^1, Psi_1^0)) Psi_2^2 = (d_x + i d_y)^2 Psi, so Im Psi_2^2 = 2 T_xy
 * and T_xy = +Im{Psi_2^2}/2; the other five entries are as printed. */
static void tidal_from_psi2(const cplx *Psi, double T[6])
{
    const cplx p20 = Psi[IX(2, 0)], p21 = Psi[IX(2, 1)], p22 = Psi[IX(2, 2)];
    T[0] = -0.5 * creal(p20) + 0.5 * creal(p22);
    T[1] = 0.5 * cimag(p22);
    T[2] = creal(p21);
    T[3] = -0.5 * creal(p20) - 0.5 * creal(p22);
    T[4] = cimag(p21);
    T[5] = creal(p20);
}

/* eq. (7) for n <= 1 (n <= 2 with T != NULL: the tidal tensor of Sec. 7.4) */
static void l2p_t(int p, const cplx *F, const double s[3], const double xb[3], double *psi, double a[3], double *T)
{
    cplx *Y = malloc(sizeof(cplx) * NCOEF(p));
    orc_upsilon(p, s[0] - xb[0], s[1] - xb[1], s[2] - xb[2], Y);
    cplx Psi[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0}; /* (n, m) for n <= 2 at IX(n, m) */
    const int nmax = T ? 2 : 1;
    for (int n = 0; n <= nmax && n <= p; ++n)
        for (int m = -n; m <= n; ++m) {
            cplx acc = 0;
            for (int k = 0; k <= p - n; ++k)
                for (int l = -k; l <= k; ++l) {
                    int nn = n + k, mm = m + l;
                    if (mm < -nn || mm > nn) continue;
                    acc += conj(Y[IX(k, l)]) * F[IX(nn, mm)];
                }
            Psi[IX(n, m)] = acc;
        }
    *psi = creal(Psi[0]);
    if (p >= 1) {
        a[0] = -creal(Psi[IX(1, 1)]);
        a[1] = -cimag(Psi[IX(1, 1)]);
        a[2] = -creal(Psi[IX(1, 0)]);
    } else {
        a[0] = a[1] = a[2] = 0.0;
    }
    if (T) {
        if (p >= 2) tidal_from_psi2(Psi, T);
        else for (int k = 0; k < 6; ++k) T[k] = 0.0;
    }
    free(Y);
}
static void l2p(int p, const cplx *F, const double s[3], const double xb[3], double *psi, double a[3])
{
    l2p_t(p, F, s, xb, psi, a, NULL);
}

/* eq. (14): P_n^2 = sum_m (n-m)! (n+m)! |M_n^m|^2 */
static void multipole_power(int p, const cplx *M, double *P)
{
    for (int n = 0; n <= p; ++n) {
        double s = 0;
        for (int m = -n; m <= n; ++m) {
            double fac = tgamma(n - m + 1.0) * tgamma(n + m + 1.0);
            double a = cabs(M[IX(n, m)]);
            s += fac * a * a;
        }
        P[n] = sqrt(s);
    }
}

/* exported single-kernel entry points for the tests (complex arrays as re/im pairs) */
static cplx *to_c(int p, const double *re, const double *im)
{
    cplx *c = malloc(sizeof(cplx) * NCOEF(p));
    for (int i = 0; i < NCOEF(p); ++i) c[i] = re[i] + I * im[i];
    return c;
}
static void from_c(int p, const cplx *c, double *re, double *im)
{
    for (int i = 0; i < NCOEF(p); ++i) { re[i] = creal(c[i]); im[i] = cimag(c[i]); }
}
void orc_p2m(int p, long n, const double *x, const double *mu, const double z[3], double *re, double *im)
{
    cplx *M = calloc(NCOEF(p), sizeof(cplx));
    p2m(p, n, x, mu, z, M);
    from_c(p, M, re, im);
    free(M);
}
void orc_m2m(int p, const double *re, const double *im, const double z[3], const double zp[3],
             double *ore, double *oim)
{
    cplx *M = to_c(p, re, im), *O = calloc(NCOEF(p), sizeof(cplx));
    m2m(p, M, z, zp, O);
    from_c(p, O, ore, oim);
    free(M); free(O);
}
void orc_m2l(int p, const double *re, const double *im, const double zA[3], const double sB[3],
             double *ore, double *oim)
{
    cplx *M = to_c(p, re, im), *O = calloc(NCOEF(p), sizeof(cplx));
    m2l(p, M, zA, sB, O);
    from_c(p, O, ore, oim);
    free(M); free(O);
}
void orc_l2l(int p, const double *re, const double *im, const double s[3], const double sp[3],
             double *ore, double *oim)
{
    cplx *F = to_c(p, re, im), *O = calloc(NCOEF(p), sizeof(cplx));
    l2l(p, F, s, sp, O);
    from_c(p, O, ore, oim);
    free(F); free(O);
}
void orc_l2p(int p, const double *re, const double *im, const double s[3], const double xb[3],
             double *psi, double a[3])
{
    cplx *F = to_c(p, re, im);
    l2p(p, F, s, xb, psi, a);
    free(F);
}
void orc_power(int p, const double *re, const double *im, double *P)
{
    cplx *M = to_c(p, re, im);
    multipole_power(p, M, P);
    free(M);
}

/* ------------------------------------------------------------------------- */
/* Rotation-accelerated M2L (App. A.5)                                        */
/* ------------------------------------------------------------------------- */

/* Swap matrix B_n of App. A.5.1 for exchanging the x and z axes:
 * Theta_n^m(z, y, x) = sum_l B_n^{ml} Theta_n^l(x, y, z).  Built from B_0 = 1 with the
 * recurrences given there, 2 B_{n+1}^{ml} = B_n^{m,l-1} - B_n^{m,l+1} for |m| <= n and
 * 2 B_{n+1}^{n+1,l} = B_n^{n,l-1} + B_n^{n,l+1} + 2 B_n^{nl},
 * 2 B_{n+1}^{-n-1,l} = B_n^{-n,l-1} + B_n^{-n,l+1} - 2 B_n^{-n,l}, entries with |l| > n
 * being zero.  B[(m+n)(2n+1) + (l+n)], row m, column l. */
static double bget(const double *b, int n, int m, int l)
{
    if (m < -n || m > n || l < -n || l > n) return 0.0;
    return b[(m + n) * (2 * n + 1) + (l + n)];
}
void orc_swap_matrix(int n, double *B)
{
    double *b = malloc(sizeof(double) * (2 * n + 1) * (2 * n + 1));
    double *nb = malloc(sizeof(double) * (2 * n + 1) * (2 * n + 1));
    b[0] = 1.0;
    for (int k = 0; k < n; ++k) {
        const int w = 2 * (k + 1) + 1;
        for (int i = 0; i < w * w; ++i) nb[i] = 0.0;
        for (int m = -k; m <= k; ++m)
            for (int l = -(k + 1); l <= k + 1; ++l)
                nb[(m + k + 1) * w + (l + k + 1)] = 0.5 * (bget(b, k, m, l - 1) - bget(b, k, m, l + 1));
        for (int l = -(k + 1); l <= k + 1; ++l) {
            nb[(2 * k + 2) * w + (l + k + 1)] = 0.5 * (bget(b, k, k, l - 1) + bget(b, k, k, l + 1) + 2.0 * bget(b, k, k, l));
            nb[0 * w + (l + k + 1)] = 0.5 * (bget(b, k, -k, l - 1) + bget(b, k, -k, l + 1) - 2.0 * bget(b, k, -k, l));
        }
        double *t = b; b = nb; nb = t;
    }
    memcpy(B, b, sizeof(double) * (2 * n + 1) * (2 * n + 1));
    free(b);
    free(nb);
}

/* X_n^m *= e^{-i m a} for every order (a rotation of the frame about z by a), e = e^{i a} */
static void rot_z(int p, cplx *X, cplx e)
{
    for (int n = 0; n <= p; ++n)
        for (int m = -n; m <= n; ++m) X[IX(n, m)] *= cpow(conj(e), m);
}
/* X_n <- S X_n per order, S = B_n (transpose = 1: B_n^T) */
static void swap_xz(int p, cplx *X, int transpose)
{
    cplx *t = malloc(sizeof(cplx) * (2 * p + 1));
    for (int n = 0; n <= p; ++n) {
        double *Bn = malloc(sizeof(double) * (2 * n + 1) * (2 * n + 1));
        orc_swap_matrix(n, Bn);
        for (int m = -n; m <= n; ++m) {
            cplx s = 0;
            for (int l = -n; l <= n; ++l)
                s += (transpose ? Bn[(l + n) * (2 * n + 1) + (m + n)] : Bn[(m + n) * (2 * n + 1) + (l + n)]) * X[IX(n, l)];
            t[m + n] = s;
        }
        for (int m = -n; m <= n; ++m) X[IX(n, m)] = t[m + n];
        free(Bn);
    }
    free(t);
}

/* eq. (3b) via rotations (App. A.5.2).  With r = s_B - z_A = (x, y, z), rho = |(x, y)|:
 * rotate the frame about z so that r lies in the y-z plane (e^{i alpha} = (y - i x)/rho),
 * swap x and z, rotate about z so that r lies on the x axis (e^{i beta} = (z + i rho)/|r|),
 * swap x and z: r is now (0, 0, |r|).  Multipoles transform with the Upsilon swap matrices
 * (B_n^T), the z-axis M2L is eq. (A31), and the local coefficients return through the
 * inverse map (the swaps B_n and the conjugate phases, in reverse order). */
static void m2l_rot(int p, const cplx *M, const double zA[3], const double sB[3], cplx *F)
{
    const double x = sB[0] - zA[0], y = sB[1] - zA[1], z = sB[2] - zA[2];
    const double rho = sqrt(x * x + y * y), R = sqrt(x * x + y * y + z * z);
    const cplx ea = rho > 0 ? (y - I * x) / rho : 1.0, eb = (z + I * rho) / R;
    cplx *Mt = malloc(sizeof(cplx) * NCOEF(p)), *Ft = malloc(sizeof(cplx) * NCOEF(p));
    memcpy(Mt, M, sizeof(cplx) * NCOEF(p));
    rot_z(p, Mt, ea);
    swap_xz(p, Mt, 1);
    rot_z(p, Mt, eb);
    swap_xz(p, Mt, 1);
    for (int n = 0; n <= p; ++n)
        for (int m = -n; m <= n; ++m) {
            cplx s = 0;
            for (int k = abs(m); k <= p - n; ++k) {
                double f = 1.0;
                for (int i = 2; i <= n + k; ++i) f *= i;
                s += sgn_m(m) * Mt[IX(k, m)] * f / pow(R, n + k + 1);
            }
            Ft[IX(n, m)] = s;
        }
    swap_xz(p, Ft, 0);
    rot_z(p, Ft, conj(eb));
    swap_xz(p, Ft, 0);
    rot_z(p, Ft, conj(ea));
    for (int i = 0; i < NCOEF(p); ++i) F[i] += Ft[i];
    free(Mt);
    free(Ft);
}
void orc_m2l_rot(int p, const double *re, const double *im, const double zA[3], const double sB[3],
                 double *ore, double *oim)
{
    cplx *M = to_c(p, re, im), *F = calloc(NCOEF(p), sizeof(cplx));
    m2l_rot(p, M, zA, sB, F);
    from_c(p, F, ore, oim);
    free(M);
    free(F);
}

/* ------------------------------------------------------------------------- */
/* Direct summation, eqs. (1) and (6), Neumaier-compensated FP64 sums          */
/* ------------------------------------------------------------------------- */

typedef struct { double s, c; } nsum;
static inline void nadd(nsum *a, double v)
{
    double t = a->s + v;
    if (fabs(a->s) >= fabs(v)) a->c += (a->s - t) + v;
    else a->c += (v - t) + a->s;
    a->s = t;
}
static inline double nval(const nsum *a) { return a->s + a->c; }

/* Psi_b = sum_{a != b} G mu_a / |x_b - x_a|, a_b = grad Psi_b, f_b = sum G mu_a / |x_b - x_a|^2,
 * for the sinks listed in `sinks` (all particles when sinks == NULL).  Pairs at distance 0
 * are skipped and counted.  Returns that count. */
long orc_direct(long n, const double *x, const double *mu, double G, long ns, const long *sinks,
                double *psi, double *acc, double *f)
{
    long coincident = 0;
    long nsink = sinks ? ns : n;
    for (long i = 0; i < nsink; ++i) {
        long b = sinks ? sinks[i] : i;
        nsum P = {0, 0}, A0 = {0, 0}, A1 = {0, 0}, A2 = {0, 0}, Fs = {0, 0};
        for (long a = 0; a < n; ++a) {
            if (a == b) continue;
            double dx = x[3 * a] - x[3 * b], dy = x[3 * a + 1] - x[3 * b + 1], dz = x[3 * a + 2] - x[3 * b + 2];
            double r2 = dx * dx + dy * dy + dz * dz;
            if (r2 == 0.0) { ++coincident; continue; }
            double r = sqrt(r2);
            double q = mu[a] / r;
            nadd(&P, q);
            double q3 = q / r2;
            nadd(&A0, q3 * dx); nadd(&A1, q3 * dy); nadd(&A2, q3 * dz);
            nadd(&Fs, mu[a] / r2);
        }
        if (psi) psi[i] = G * nval(&P);
        if (acc) { acc[3 * i] = G * nval(&A0); acc[3 * i + 1] = G * nval(&A1); acc[3 * i + 2] = G * nval(&A2); }
        if (f) f[i] = G * nval(&Fs);
    }
    return coincident;
}

/* the tidal tensor T = grad grad Psi of eq. (1) at the sinks (Sec. 7.4), directly:
 * T_b = sum_a G mu_a (3 d d^T - r^2 I) / r^5 with d = x_b - x_a, as (xx, xy, xz, yy, yz, zz) */
void orc_direct_tidal(long n, const double *x, const double *mu, double G, long ns, const long *sinks, double *T)
{
    long nsink = sinks ? ns : n;
    for (long i = 0; i < nsink; ++i) {
        long b = sinks ? sinks[i] : i;
        nsum S[6] = {{0, 0}, {0, 0}, {0, 0}, {0, 0}, {0, 0}, {0, 0}};
        for (long a = 0; a < n; ++a) {
            if (a == b) continue;
            double d[3] = {x[3 * b] - x[3 * a], x[3 * b + 1] - x[3 * a + 1], x[3 * b + 2] - x[3 * a + 2]};
            double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
            if (r2 == 0.0) continue;
            double r = sqrt(r2), q5 = mu[a] / (r2 * r2 * r);
            int k = 0;
            for (int u = 0; u < 3; ++u)
                for (int v = u; v < 3; ++v) nadd(&S[k++], q5 * (3.0 * d[u] * d[v] - (u == v ? r2 : 0.0)));
        }
        for (int k = 0; k < 6; ++k) T[6 * i + k] = G * nval(&S[k]);
    }
}

/* ------------------------------------------------------------------------- */
/* Smallest enclosing balls (Sec. 5.1.1; reading R-ses)                       */
/* ------------------------------------------------------------------------- */

/* The balls are computed in IEEE single precision in coordinates relative to a
 * reference point of the cell (its first particle, or its first daughter's
 * centre); the centre is converted back to FP64 and the radius rho is then
 * recomputed exactly in FP64 over the cell's particles (Sec. 4), so the
 * single-precision ball only decides where the expansion centre sits.
 * Tolerances: support sets are singular below 1e-6 of the Gram scale, a point
 * or ball counts as inside within a relative 1e-5 of the radius. */
#define MEB_SING 1e-6f
#define MEB_IN 1e-5f

/* Solve a k x k symmetric system (k <= 3) with two right-hand sides by Gaussian
 * elimination with partial pivoting.  Returns 0 when (numerically) singular. */
static int solve_small(int k, float A[3][3], float b[2][3], float x[2][3])
{
    float M[3][5];
    float scale = 0;
    for (int i = 0; i < k; ++i)
        for (int j = 0; j < k; ++j) if (fabsf(A[i][j]) > scale) scale = fabsf(A[i][j]);
    if (scale == 0) return 0;
    for (int i = 0; i < k; ++i) {
        for (int j = 0; j < k; ++j) M[i][j] = A[i][j];
        M[i][k] = b[0][i];
        M[i][k + 1] = b[1][i];
    }
    for (int c = 0; c < k; ++c) {
        int piv = c;
        for (int r = c + 1; r < k; ++r) if (fabsf(M[r][c]) > fabsf(M[piv][c])) piv = r;
        if (fabsf(M[piv][c]) <= MEB_SING * scale) return 0;
        if (piv != c) for (int j = 0; j < k + 2; ++j) { float t = M[c][j]; M[c][j] = M[piv][j]; M[piv][j] = t; }
        for (int r = c + 1; r < k; ++r) {
            float fct = M[r][c] / M[c][c];
            for (int j = c; j < k + 2; ++j) M[r][j] -= fct * M[c][j];
        }
    }
    for (int rhs = 0; rhs < 2; ++rhs)
        for (int r = k - 1; r >= 0; --r) {
            float s = M[r][k + rhs];
            for (int j = r + 1; j < k; ++j) s -= M[r][j] * x[rhs][j];
            x[rhs][r] = s / M[r][r];
        }
    return 1;
}

/* The smallest ball whose boundary touches every ball of the support set
 * {(c_i, r_i)} from inside (|c - c_i| + r_i = R), with its centre in the affine hull
 * of the c_i: with u = c - c_0 = sum_j lam_j d_j, d_j = c_j - c_0, the tangency
 * conditions give G lam = a + R b (G the Gram matrix of the d_j,
 * a_j = (|d_j|^2 - r_j^2 + r_0^2)/2, b_j = r_j - r_0) and |u| = R - r_0 a quadratic
 * in R.  With all r_i = 0 it is the circumsphere through the points.
 * Returns 0 if there is no such ball (degenerate support set). */
static int support_ball(int k, const float c[][3], const float *r, float out_c[3], float *out_r)
{
    if (k == 1) {
        for (int d = 0; d < 3; ++d) out_c[d] = c[0][d];
        *out_r = r[0];
        return 1;
    }
    int q = k - 1;
    float D[3][3], G[3][3], rhs[2][3], sol[2][3];
    for (int j = 0; j < q; ++j)
        for (int d = 0; d < 3; ++d) D[j][d] = c[j + 1][d] - c[0][d];
    for (int i = 0; i < q; ++i) {
        for (int j = 0; j < q; ++j) G[i][j] = D[i][0] * D[j][0] + D[i][1] * D[j][1] + D[i][2] * D[j][2];
        rhs[0][i] = 0.5f * (G[i][i] - r[i + 1] * r[i + 1] + r[0] * r[0]);
        rhs[1][i] = r[i + 1] - r[0];
    }
    if (!solve_small(q, G, rhs, sol)) return 0;
    float A[3] = {0, 0, 0}, B[3] = {0, 0, 0};
    for (int j = 0; j < q; ++j)
        for (int d = 0; d < 3; ++d) { A[d] += sol[0][j] * D[j][d]; B[d] += sol[1][j] * D[j][d]; }
    float qa = B[0] * B[0] + B[1] * B[1] + B[2] * B[2] - 1.0f;
    float qb = A[0] * B[0] + A[1] * B[1] + A[2] * B[2] + r[0];
    float qc = A[0] * A[0] + A[1] * A[1] + A[2] * A[2] - r[0] * r[0];
    float rmax = r[0];
    for (int i = 1; i < k; ++i) if (r[i] > rmax) rmax = r[i];
    float R = -1.0f;
    if (fabsf(qa) < 1e-6f) {
        if (qb == 0) return 0;
        R = -qc / (2.0f * qb);
    } else {
        float disc = qb * qb - qa * qc;
        if (disc < 0) {
            if (disc < -MEB_SING * (qb * qb + fabsf(qa * qc))) return 0;
            disc = 0;
        }
        float sq = sqrtf(disc);
        float r1 = (-qb - sq) / qa, r2 = (-qb + sq) / qa;
        float lo = r1 < r2 ? r1 : r2, hi = r1 < r2 ? r2 : r1;
        float tol = MEB_SING * fabsf(rmax);
        if (lo >= rmax - tol) R = lo;
        else if (hi >= rmax - tol) R = hi;
        else return 0;
    }
    if (!(R >= 0) || R < rmax - MEB_SING * rmax) return 0;
    for (int d = 0; d < 3; ++d) out_c[d] = c[0][d] + A[d] + R * B[d];
    *out_r = R;
    return 1;
}

static inline float dist3f(const float a[3], const float b[3])
{
    float dx = a[0] - b[0], dy = a[1] - b[1], dz = a[2] - b[2];
    return sqrtf(dx * dx + dy * dy + dz * dz);
}
static inline double dist3(const double a[3], const double b[3])
{
    double dx = a[0] - b[0], dy = a[1] - b[1], dz = a[2] - b[2];
    return sqrt(dx * dx + dy * dy + dz * dz);
}

/* smallest ball with all support points on its boundary (Welzl's b_md(empty, R)) */
static void trivial_ball(int nr, const float R[][3], float c[3], float *rad)
{
    const float zr[4] = {0, 0, 0, 0};
    if (nr == 0) { c[0] = c[1] = c[2] = 0; *rad = -1.0f; return; }
    if (support_ball(nr, R, zr, c, rad)) return;
    /* degenerate support set: the smallest ball through a subset that still
     * contains every support point */
    float best = -1;
    for (int mask = 1; mask < (1 << nr); ++mask) {
        float sub[4][3]; int k = 0;
        for (int i = 0; i < nr; ++i) if (mask & (1 << i)) { for (int d = 0; d < 3; ++d) sub[k][d] = R[i][d]; ++k; }
        float cc[3], rr;
        if (!support_ball(k, sub, zr, cc, &rr)) continue;
        int ok = 1;
        for (int i = 0; i < nr; ++i) if (dist3f(R[i], cc) > rr * (1.0f + MEB_IN)) { ok = 0; break; }
        if (ok && (best < 0 || rr < best)) { best = rr; c[0] = cc[0]; c[1] = cc[1]; c[2] = cc[2]; *rad = rr; }
    }
}

static inline int in_ball(const float pt[3], const float c[3], float rad)
{
    if (rad < 0) return 0;
    return dist3f(pt, c) <= rad * (1.0f + MEB_IN);
}

/* Welzl's recursion: the smallest ball enclosing P[0..np) with R on its boundary */
static void welzl(int np, const float P[][3], int nr, float R[4][3], float c[3], float *rad)
{
    if (np == 0 || nr == 4) { trivial_ball(nr, (const float(*)[3])R, c, rad); return; }
    welzl(np - 1, P, nr, R, c, rad);
    if (in_ball(P[np - 1], c, *rad)) return;
    for (int d = 0; d < 3; ++d) R[nr][d] = P[np - 1][d];
    welzl(np - 1, P, nr + 1, R, c, rad);
}

/* The order in which Welzl's recursion takes the points (reading R-ses): the first
 * min(n, 128) points in bit-reversed index order, i.e. t = 0, 1, 2, ... over the
 * smallest power of two K >= min(n, 128), taking bitreverse_K(t) whenever it is
 * below min(n, 128); any further points in index order.  Points of a leaf come in
 * key order, which is spatially coherent and makes the recursion restart often;
 * the bit-reversed order visits them spread out.  The ball is the same (it is
 * unique); only the work changes. */
static void meb_order(int n, int *order)
{
    int m = n < 128 ? n : 128, K = 1, bits = 0, k = 0;
    while (K < m) { K <<= 1; ++bits; }
    for (int t = 0; t < K; ++t) {
        int v = 0;
        for (int b = 0; b < bits; ++b) if (t & (1 << b)) v |= 1 << (bits - 1 - b);
        if (v < m) order[k++] = v;
    }
    for (int i = m; i < n; ++i) order[k++] = i;
}

/* Welzl's recursion with the move-to-front rule (Gaertner): the smallest ball
 * enclosing L[0..end) with R on its boundary; a point found outside is moved to the
 * front of L after the recursion it starts, so later scans meet it first.  Used for
 * up to 128 points (reading R-ses). */
static void welzl_mtf(int end, float (*L)[3], int nr, float R[4][3], float c[3], float *rad)
{
    trivial_ball(nr, (const float(*)[3])R, c, rad);
    if (nr == 4) return;
    for (int i = 0; i < end; ++i) {
        if (in_ball(L[i], c, *rad)) continue;
        for (int d = 0; d < 3; ++d) R[nr][d] = L[i][d];
        welzl_mtf(i, L, nr + 1, R, c, rad);
        float t[3] = {L[i][0], L[i][1], L[i][2]};
        for (int j = i; j > 0; --j)
            for (int d = 0; d < 3; ++d) L[j][d] = L[j - 1][d];
        for (int d = 0; d < 3; ++d) L[0][d] = t[d];
    }
}

/* smallest enclosing ball of n points: single precision, relative to the first point */
int orc_meb_points(int n, const double *pts, double c[3], double *rad)
{
    if (n <= 0) { c[0] = c[1] = c[2] = 0; *rad = 0; return 0; }
    float (*P)[3] = malloc(sizeof(float[3]) * n);
    int *order = malloc(sizeof(int) * n);
    meb_order(n, order);
    for (int i = 0; i < n; ++i)
        for (int d = 0; d < 3; ++d) P[i][d] = (float)(pts[3 * order[i] + d] - pts[d]);
    free(order);
    float R[4][3], cf[3], rf;
    if (n <= 128) welzl_mtf(n, P, 0, R, cf, &rf);
    else welzl(n, (const float(*)[3])P, 0, R, cf, &rf);
    free(P);
    for (int d = 0; d < 3; ++d) c[d] = pts[d] + (double)cf[d];
    *rad = rf < 0 ? 0.0 : (double)rf;
    return 1;
}

/* smallest ball enclosing n <= 8 balls: the smallest, over all support sets of 1..4
 * balls (enumerated by bit mask), of the support balls that contain every ball;
 * single precision, relative to the first ball's centre */
int orc_meb_balls(int n, const double *cen, const double *radii, double c[3], double *rad)
{
    float C[8][3], Rr[8];
    for (int i = 0; i < n; ++i) {
        for (int d = 0; d < 3; ++d) C[i][d] = (float)(cen[3 * i + d] - cen[d]);
        Rr[i] = (float)radii[i];
    }
    float best = -1, bc[3] = {0, 0, 0};
    for (int mask = 1; mask < (1 << n); ++mask) {
        int k = 0; float sc[4][3], sr[4];
        for (int i = 0; i < n && k <= 4; ++i)
            if (mask & (1 << i)) {
                if (k == 4) { k = 5; break; }
                for (int d = 0; d < 3; ++d) sc[k][d] = C[i][d];
                sr[k] = Rr[i];
                ++k;
            }
        if (k > 4) continue;
        float cc[3], rr;
        if (!support_ball(k, (const float(*)[3])sc, sr, cc, &rr)) continue;
        int ok = 1;
        for (int i = 0; i < n; ++i)
            if (dist3f(C[i], cc) + Rr[i] > rr * (1.0f + MEB_IN)) { ok = 0; break; }
        if (ok && (best < 0 || rr < best)) { best = rr; bc[0] = cc[0]; bc[1] = cc[1]; bc[2] = cc[2]; }
    }
    if (best < 0) return 0;
    for (int d = 0; d < 3; ++d) c[d] = cen[d] + (double)bc[d];
    *rad = (double)best;
    return 1;
}

/* ------------------------------------------------------------------------- */
/* The oct-tree (Sec. 2.2; readings R-box, R-key, R-leaf)                     */
/* ------------------------------------------------------------------------- */

#define MAXLEVEL 21

typedef struct {
    int level, leaf;
    long first, count;       /* particle range in sorted order */
    long child, nchild;      /* first daughter index, number of daughters */
    double s[3], rho, mass;  /* centre z = s (smallest enclosing sphere), radius, mass */
    double com[3], rho_com;  /* centre of mass and its radius (low-order estimator) */
    double minscale;         /* min over the cell's sinks of the acceleration scale */
    long nactive;            /* active particles in the cell (Sec. 7.1; all when no subset) */
} cell_t;

typedef struct {
    long n;
    double *xs, *mus;     /* sorted positions [n][3] and masses */
    long *perm;           /* perm[i] = original index of sorted particle i */
    unsigned char *act;   /* act[i]: sorted particle i is an active sink (Sec. 7.1) */
    uint64_t *keys;
    cell_t *cells;
    long ncells, cap;
    int leaf_size;
    double lo[3], side;
} tree_t;

typedef struct { uint64_t key; long idx; } keyidx;
static int cmp_keyidx(const void *a, const void *b)
{
    const keyidx *u = a, *v = b;
    if (u->key != v->key) return u->key < v->key ? -1 : 1;
    return (u->idx > v->idx) - (u->idx < v->idx);
}

static uint64_t morton_key(const double x[3], const double lo[3], double side)
{
    uint32_t q[3];
    for (int d = 0; d < 3; ++d) {
        double t = (x[d] - lo[d]) / side;
        double u = t * 2097152.0; /* 2^21 */
        long v = (long)floor(u);
        if (v < 0) v = 0;
        if (v > 2097151) v = 2097151;
        q[d] = (uint32_t)v;
    }
    uint64_t key = 0;
    for (int b = MAXLEVEL - 1; b >= 0; --b)
        key = (key << 3) | ((uint64_t)((q[0] >> b) & 1) << 2) | ((uint64_t)((q[1] >> b) & 1) << 1) |
              (uint64_t)((q[2] >> b) & 1);
    return key;
}

static long new_cell(tree_t *t)
{
    if (t->ncells == t->cap) {
        t->cap = t->cap ? 2 * t->cap : 1024;
        t->cells = realloc(t->cells, sizeof(cell_t) * t->cap);
    }
    memset(&t->cells[t->ncells], 0, sizeof(cell_t));
    return t->ncells++;
}

static void split_cell(tree_t *t, long ci)
{
    cell_t c = t->cells[ci];
    if (c.count <= t->leaf_size || c.level >= MAXLEVEL) { t->cells[ci].leaf = 1; return; }
    int shift = 3 * (MAXLEVEL - (c.level + 1));
    long bounds[9];
    long pos = c.first;
    for (int o = 0; o < 8; ++o) {
        bounds[o] = pos;
        while (pos < c.first + c.count && (long)((t->keys[pos] >> shift) & 7) == o) ++pos;
    }
    bounds[8] = c.first + c.count;
    int nonempty = 0;
    for (int o = 0; o < 8; ++o) if (bounds[o + 1] > bounds[o]) ++nonempty;
    long first_child = t->ncells;
    for (int k = 0; k < nonempty; ++k) new_cell(t);
    int k = 0;
    for (int o = 0; o < 8; ++o) {
        if (bounds[o + 1] == bounds[o]) continue;
        cell_t *d = &t->cells[first_child + k];
        d->level = c.level + 1;
        d->first = bounds[o];
        d->count = bounds[o + 1] - bounds[o];
        ++k;
    }
    t->cells[ci].leaf = 0;
    t->cells[ci].child = first_child;
    t->cells[ci].nchild = nonempty;
    for (int j = 0; j < nonempty; ++j) split_cell(t, first_child + j);
}

static void build_tree(tree_t *t, long n, const double *x, const double *mu, int leaf_size)
{
    memset(t, 0, sizeof(*t));
    t->n = n;
    t->leaf_size = leaf_size;
    double lo[3] = {x[0], x[1], x[2]}, hi[3] = {x[0], x[1], x[2]};
    for (long i = 1; i < n; ++i)
        for (int d = 0; d < 3; ++d) {
            if (x[3 * i + d] < lo[d]) lo[d] = x[3 * i + d];
            if (x[3 * i + d] > hi[d]) hi[d] = x[3 * i + d];
        }
    double ext = 0;
    for (int d = 0; d < 3; ++d) if (hi[d] - lo[d] > ext) ext = hi[d] - lo[d];
    double side = ext * (1.0 + 0x1p-20);
    if (!(side > 0)) side = 1.0;
    for (int d = 0; d < 3; ++d) t->lo[d] = lo[d];
    t->side = side;
    keyidx *ki = malloc(sizeof(keyidx) * n);
    for (long i = 0; i < n; ++i) { ki[i].key = morton_key(&x[3 * i], lo, side); ki[i].idx = i; }
    qsort(ki, n, sizeof(keyidx), cmp_keyidx);
    t->xs = malloc(sizeof(double) * 3 * n);
    t->mus = malloc(sizeof(double) * n);
    t->perm = malloc(sizeof(long) * n);
    t->keys = malloc(sizeof(uint64_t) * n);
    for (long i = 0; i < n; ++i) {
        long j = ki[i].idx;
        t->perm[i] = j;
        t->keys[i] = ki[i].key;
        for (int d = 0; d < 3; ++d) t->xs[3 * i + d] = x[3 * j + d];
        t->mus[i] = mu[j];
    }
    free(ki);
    long root = new_cell(t);
    t->cells[root].level = 0;
    t->cells[root].first = 0;
    t->cells[root].count = n;
    split_cell(t, root);
}

static void free_tree(tree_t *t)
{
    free(t->xs); free(t->mus); free(t->perm); free(t->act); free(t->keys); free(t->cells);
    memset(t, 0, sizeof(*t));
}

/* centres and radii, bottom-up (reading R-ses), plus mass and centre of mass */
/* keep_centre: a re-cycled tree (Sec. 7.1) keeps the centres s and recomputes the radii,
 * masses and centres of mass for the particles' current positions */
static void cell_geometry_k(tree_t *t, long ci, int keep_centre)
{
    cell_t *c = &t->cells[ci];
    if (!c->leaf)
        for (long j = 0; j < c->nchild; ++j) cell_geometry_k(t, c->child + j, keep_centre);
    c = &t->cells[ci];
    const double *X = &t->xs[3 * c->first];
    if (keep_centre) {
        /* s stays */
    } else if (c->leaf) {
        orc_meb_points((int)c->count, X, c->s, &c->rho);
    } else {
        double cen[8 * 3], rad[8];
        for (long j = 0; j < c->nchild; ++j) {
            cell_t *d = &t->cells[c->child + j];
            for (int k = 0; k < 3; ++k) cen[3 * j + k] = d->s[k];
            rad[j] = d->rho;
        }
        if (!orc_meb_balls((int)c->nchild, cen, rad, c->s, &c->rho))
            for (int k = 0; k < 3; ++k) c->s[k] = cen[k]; /* no valid support set: first daughter's centre */
    }
    double rmax = 0, m = 0, mx[3] = {0, 0, 0};
    for (long i = 0; i < c->count; ++i) {
        double r = dist3(&X[3 * i], c->s);
        if (r > rmax) rmax = r;
        double w = t->mus[c->first + i];
        m += w;
        for (int k = 0; k < 3; ++k) mx[k] += w * X[3 * i + k];
    }
    c->rho = rmax;
    c->mass = m;
    for (int k = 0; k < 3; ++k) c->com[k] = (m > 0) ? mx[k] / m : c->s[k];
    double rc = 0;
    for (long i = 0; i < c->count; ++i) {
        double r = dist3(&X[3 * i], c->com);
        if (r > rc) rc = r;
    }
    c->rho_com = rc;
}
static void cell_geometry(tree_t *t, long ci) { cell_geometry_k(t, ci, 0); }

/* ------------------------------------------------------------------------- */
/* Dual tree walk (Sec. 2.2.2) and acceptance criteria (eqs. 9, 15-18)        */
/* ------------------------------------------------------------------------- */

typedef struct { long a, b; int q; } pair_t;  /* q: the M2L interaction's expansion order */
typedef struct { pair_t *v; long n, cap; } plist;
static void push_q(plist *l, long a, long b, int q)
{
    if (l->n == l->cap) { l->cap = l->cap ? 2 * l->cap : 4096; l->v = realloc(l->v, sizeof(pair_t) * l->cap); }
    l->v[l->n].a = a; l->v[l->n].b = b; l->v[l->n].q = q; ++l->n;
}
static void push(plist *l, long a, long b) { push_q(l, a, b, 0); }

enum { MAC_A = 0, MAC_F = 1, MAC_THETA = 2, MAC_EST = 3 };

typedef struct {
    const tree_t *t;
    int p, mac, use_com;
    double eps, theta_crit, p2p_thresh;
    const double *P;      /* multipole power [ncells][p+1] (MAC_A/MAC_F) */
    int adaptive;         /* per-interaction order (Sec. 7, opening) */
    plist m2l, p2p;
} walk_t;

/* E~_{A->B} M_A / r^2 of order q, eqs. (15)-(17), without the division by M_A:
 * M_A E_{A->B} = sum_k C(q,k) P_k rho_B^{q-k} / r^q (eq. 15; P_k of eq. 14 for the source
 * cell A, P_0 = M_A), times 8 max(rho_A, rho_B) / (rho_A + rho_B) (eq. 17), over r^2.
 * The one function behind every acceptance decision of the oracle's walk. */
double orc_mac_lhs(int q, const double *P, double r, double ra, double rb)
{
    double sum = 0, cqk = 1.0;  /* C(q, k), exact integers for q <= 20 */
    for (int k = 0; k <= q; ++k) {
        sum += cqk * (P[k] / pow(r, k)) * pow(rb / r, q - k);
        cqk = cqk * (q - k) / (k + 1);
    }
    double mx = ra > rb ? ra : rb;
    double fac = (ra + rb > 0) ? 8.0 * mx / (ra + rb) : 8.0;
    return fac * sum / (r * r);
}

/* 0: not accepted; else the order of the accepted M2L interaction: p, or with the adaptive
 * walk the lowest q in [min(3, p), p] whose estimate of order q passes as well */
static int accept(const walk_t *w, long A, long B)
{
    const cell_t *a = &w->t->cells[A], *b = &w->t->cells[B];
    const double *za = w->use_com ? a->com : a->s, *sb = w->use_com ? b->com : b->s;
    double ra = w->use_com ? a->rho_com : a->rho, rb = w->use_com ? b->rho_com : b->rho;
    double r = dist3(sb, za);
    double theta = (ra + rb) / r;           /* eq. (9) */
    if (w->mac == MAC_THETA) return theta < w->theta_crit ? w->p : 0;
    if (!(theta < 1.0)) return 0;
    if (w->mac == MAC_EST) return w->p > 0 ? w->p : 1;
    /* E~_{A->B} M_A / r^2, eqs. (15)-(17), without the division by M_A */
    const double *P = &w->P[(long)A * (w->p + 1)];
    const double lhs = orc_mac_lhs(w->p, P, r, ra, rb);
    const double rhs = w->eps * b->minscale;
    if (!(lhs < rhs)) return 0;             /* eqs. (18a) / (18b) */
    if (w->adaptive)
        for (int q = w->p < 3 ? w->p : 3; q < w->p; ++q)
            if (orc_mac_lhs(q, P, r, ra, rb) < rhs) return q;
    return w->p;
}

static void walk(walk_t *w, long A, long B)
{
    const cell_t *a = &w->t->cells[A], *b = &w->t->cells[B];
    if (!b->nactive) return;  /* Sec. 7.1: only sink cells holding an active particle */
    if ((double)a->count * (double)b->count < w->p2p_thresh) { push(&w->p2p, A, B); return; }
    if (A == B) {
        if (a->leaf) { push(&w->p2p, A, B); return; }
        for (long i = 0; i < a->nchild; ++i)
            for (long j = 0; j < a->nchild; ++j) walk(w, a->child + i, a->child + j);
        return;
    }
    int q = accept(w, A, B);
    if (q) { push_q(&w->m2l, A, B, q); return; }
    if (a->leaf && b->leaf) { push(&w->p2p, A, B); return; }
    double ra = w->use_com ? a->rho_com : a->rho, rb = w->use_com ? b->rho_com : b->rho;
    int split_a = (ra >= rb);
    if (a->leaf) split_a = 0;
    if (b->leaf) split_a = 1;
    if (split_a) for (long i = 0; i < a->nchild; ++i) walk(w, a->child + i, B);
    else for (long j = 0; j < b->nchild; ++j) walk(w, A, b->child + j);
}

/* P2P over a cell pair (eq. 1): all particles of A act on all particles of B */
static void p2p_pair(const tree_t *t, long A, long B, double *psi, double *acc, long *coincident, int want_f)
{
    const cell_t *a = &t->cells[A], *b = &t->cells[B];
    for (long i = b->first; i < b->first + b->count; ++i) {
        double P = 0, ax = 0, ay = 0, az = 0;
        for (long j = a->first; j < a->first + a->count; ++j) {
            if (i == j) continue;
            double dx = t->xs[3 * j] - t->xs[3 * i], dy = t->xs[3 * j + 1] - t->xs[3 * i + 1],
                   dz = t->xs[3 * j + 2] - t->xs[3 * i + 2];
            double r2 = dx * dx + dy * dy + dz * dz;
            if (r2 == 0.0) { ++*coincident; continue; }
            if (want_f) { P += t->mus[j] / r2; continue; }
            double r = sqrt(r2);
            double q = t->mus[j] / r;
            P += q;
            double q3 = q / r2;
            ax += q3 * dx; ay += q3 * dy; az += q3 * dz;
        }
        psi[i] += P;
        if (!want_f) { acc[3 * i] += ax; acc[3 * i + 1] += ay; acc[3 * i + 2] += az; }
    }
}

/* the near-field part of the tidal tensor over a cell pair: T_i += mu_j (3 d d^T - r^2 I)/r^5 */
static void p2p_tidal_pair(const tree_t *t, long A, long B, double *T)
{
    const cell_t *a = &t->cells[A], *b = &t->cells[B];
    for (long i = b->first; i < b->first + b->count; ++i) {
        double S[6] = {0, 0, 0, 0, 0, 0};
        for (long j = a->first; j < a->first + a->count; ++j) {
            if (i == j) continue;
            double d[3] = {t->xs[3 * i] - t->xs[3 * j], t->xs[3 * i + 1] - t->xs[3 * j + 1],
                           t->xs[3 * i + 2] - t->xs[3 * j + 2]};
            double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
            if (r2 == 0.0) continue;
            double r = sqrt(r2), q5 = t->mus[j] / (r2 * r2 * r);
            int k = 0;
            for (int u = 0; u < 3; ++u)
                for (int v = u; v < 3; ++v) S[k++] += q5 * (3.0 * d[u] * d[v] - (u == v ? r2 : 0.0));
        }
        for (int k = 0; k < 6; ++k) T[6 * i + k] += S[k];
    }
}

/* ------------------------------------------------------------------------- */
/* Whole evaluation                                                           */
/* ------------------------------------------------------------------------- */

typedef struct {
    int p;            /* expansion order, 1..20 */
    double eps;       /* accuracy parameter of eqs. (18) */
    int mac;          /* 0: (18a) with a-scale, 1: (18b) with f-scale, 2: theta < theta_crit */
    double theta_crit;
    int leaf_size;
    double p2p_c;     /* direct summation when N_A N_B < p2p_c p^3 */
    int scale_src;    /* 0: low-order FMM estimate, 1: caller-supplied per-particle scale */
    int want_tidal;   /* 1: also the tidal tensor of Sec. 7.4 */
    int adaptive_p;   /* 1: per-interaction order (Sec. 7, opening) */
} orc_params;

typedef struct {
    long ncells, nleaves, n_m2l, n_p2p, p2p_interactions, coincident, est_m2l, est_p2p;
    int depth;
} orc_stats;

typedef struct {
    tree_t t;
    orc_params prm;
    plist m2l, p2p;
    double *scale_sorted; /* per sorted particle: the scale used in the MAC */
    double *psi, *acc;    /* caller order, G applied */
    double *tidal;        /* caller order [n][6] (xx, xy, xz, yy, yz, zz), G applied; NULL unless asked */
    orc_stats st;
} orc_run;

/* low-order FMM estimate of |a_b| (p = 1, eq. 18a) or f_b (p = 0, eq. 18b) with
 * theta < 1 and z = s = centre of mass (Sec. 5.3.2); output in sorted order */
static void estimate_scale(orc_run *run, int want_f, double *scale)
{
    tree_t *t = &run->t;
    int pe = want_f ? 0 : 1;
    long nc = t->ncells, n = t->n;
    int nco = NCOEF(pe);
    cplx *M = calloc((size_t)nc * nco, sizeof(cplx));
    cplx *F = calloc((size_t)nc * nco, sizeof(cplx));
    /* multipoles about the centre of mass; for p = 0 only the mass is needed */
    for (long ci = nc - 1; ci >= 0; --ci) {
        cell_t *c = &t->cells[ci];
        if (c->leaf) p2m(pe, c->count, &t->xs[3 * c->first], &t->mus[c->first], c->com, &M[ci * nco]);
        else
            for (long j = 0; j < c->nchild; ++j)
                m2m(pe, &M[(c->child + j) * nco], t->cells[c->child + j].com, c->com, &M[ci * nco]);
    }
    walk_t w = {0};
    w.t = t; w.p = pe; w.mac = MAC_EST; w.use_com = 1;
    /* reading R-p2p: the threshold uses the order of the expansion in use, here pe */
    w.p2p_thresh = run->prm.p2p_c * pow((double)pe, 3);
    walk(&w, 0, 0);
    run->st.est_m2l = w.m2l.n; run->st.est_p2p = w.p2p.n;
    for (long i = 0; i < w.m2l.n; ++i) {
        long A = w.m2l.v[i].a, B = w.m2l.v[i].b;
        if (want_f) {
            /* the 1/r^2 kernel at lowest order: F = M_A / |s_B - z_A|^2 */
            double r = dist3(t->cells[B].com, t->cells[A].com);
            F[B * nco] += t->cells[A].mass / (r * r);
        } else {
            m2l(pe, &M[A * nco], t->cells[A].com, t->cells[B].com, &F[B * nco]);
        }
    }
    double *ps = calloc(n, sizeof(double)), *ac = calloc(3 * n, sizeof(double));
    long coin = 0;
    for (long i = 0; i < w.p2p.n; ++i) p2p_pair(t, w.p2p.v[i].a, w.p2p.v[i].b, ps, ac, &coin, want_f);
    /* pass down and evaluate */
    for (long ci = 0; ci < nc; ++ci) {
        cell_t *c = &t->cells[ci];
        if (!c->leaf) {
            for (long j = 0; j < c->nchild; ++j) {
                long d = c->child + j;
                if (want_f) F[d * nco] += F[ci * nco];
                else l2l(pe, &F[ci * nco], c->com, t->cells[d].com, &F[d * nco]);
            }
        } else {
            for (long i = c->first; i < c->first + c->count; ++i) {
                if (want_f) { scale[i] = creal(F[ci * nco]) + ps[i]; continue; }
                double psi_l, a[3];
                l2p(pe, &F[ci * nco], c->com, &t->xs[3 * i], &psi_l, a);
                double gx = a[0] + ac[3 * i], gy = a[1] + ac[3 * i + 1], gz = a[2] + ac[3 * i + 2];
                scale[i] = sqrt(gx * gx + gy * gy + gz * gz);
            }
        }
    }
    free(ps); free(ac); free(M); free(F); free(w.m2l.v); free(w.p2p.v);
}

static void min_scale(tree_t *t, long ci, const double *scale)
{
    cell_t *c = &t->cells[ci];
    double m = INFINITY;
    if (c->leaf) {
        for (long i = c->first; i < c->first + c->count; ++i)
            if (t->act[i] && scale[i] < m) m = scale[i];  /* over the active sinks */
    } else {
        for (long j = 0; j < c->nchild; ++j) {
            min_scale(t, c->child + j, scale);
            if (t->cells[c->child + j].minscale < m) m = t->cells[c->child + j].minscale;
        }
    }
    t->cells[ci].minscale = m;
}

static int depth_of(const tree_t *t)
{
    int d = 0;
    for (long i = 0; i < t->ncells; ++i) if (t->cells[i].level > d) d = t->cells[i].level;
    return d;
}

void orc_run_free(orc_run *run);

static void evaluate_on_tree(orc_run *run, double G, const double *scale_in, const unsigned char *active,
                             const double *eps_b);

/* The whole FMM (Sec. 2.2.2): returns NULL on invalid input. */
/* Sec. 7.1: active (caller order, may be NULL = all) marks the sinks whose forces are
 * computed; all particles are sources.  Sink cells without an active particle take part
 * in no interaction; the MAC scale of a cell is the minimum over its active particles;
 * psi and acc of inactive particles are NaN. */
orc_run *orc_fmm_active(long n, const double *x, const double *mu, double G, const orc_params *prm,
                        const double *scale_in /* caller order, may be NULL */,
                        const unsigned char *active /* caller order, may be NULL */,
                        const double *eps_b /* caller order, may be NULL */)
{
    if (n < 0 || !prm || prm->p < 1 || prm->p > 20 || prm->leaf_size < 1) return NULL;
    if (prm->mac != MAC_THETA && !(prm->eps > 0)) return NULL;
    for (long i = 0; i < n; ++i) {
        if (!isfinite(x[3 * i]) || !isfinite(x[3 * i + 1]) || !isfinite(x[3 * i + 2]) ||
            !isfinite(mu[i]) || mu[i] < 0)
            return NULL;
    }
    orc_run *run = calloc(1, sizeof(orc_run));
    run->prm = *prm;
    run->psi = calloc(n > 0 ? n : 1, sizeof(double));
    run->acc = calloc(3 * (n > 0 ? n : 1), sizeof(double));
    if (n == 0) return run;
    tree_t *t = &run->t;
    build_tree(t, n, x, mu, prm->leaf_size);
    cell_geometry(t, 0);
    evaluate_on_tree(run, G, scale_in, active, eps_b);
    return run;
}

/* everything after the tree and its geometry (shared by fresh and re-cycled trees) */
static void evaluate_on_tree(orc_run *run, double G, const double *scale_in, const unsigned char *active,
                             const double *eps_b)
{
    const orc_params *prm = &run->prm;
    tree_t *t = &run->t;
    const long n = t->n;
    int p = prm->p, nco = NCOEF(p);
    long nc = t->ncells;
    free(t->act);
    t->act = malloc(n);
    for (long i = 0; i < n; ++i) t->act[i] = active ? (active[t->perm[i]] != 0) : 1;
    for (long ci = 0; ci < nc; ++ci) {
        cell_t *c = &t->cells[ci];
        c->nactive = 0;
        for (long i = c->first; i < c->first + c->count; ++i) c->nactive += t->act[i];
    }
    run->st.ncells = nc;
    for (long i = 0; i < nc; ++i) run->st.nleaves += t->cells[i].leaf;
    run->st.depth = depth_of(t);

    /* acceleration scale for the MAC */
    run->scale_sorted = calloc(n, sizeof(double));
    if (prm->mac == MAC_A || prm->mac == MAC_F) {
        if (prm->scale_src == 1 && scale_in) {
            for (long i = 0; i < n; ++i) run->scale_sorted[i] = scale_in[t->perm[i]];
        } else {
            estimate_scale(run, prm->mac == MAC_F, run->scale_sorted);
        }
        /* individual accuracy parameters (Sec. 7, opening): the criterion's right-hand side
         * becomes min_{b in B} eps_b a_b, i.e. eps times the minimum of (eps_b / eps) a_b */
        if (eps_b)
            for (long i = 0; i < n; ++i) run->scale_sorted[i] *= eps_b[t->perm[i]] / prm->eps;
        min_scale(t, 0, run->scale_sorted);
    }

    /* upward pass: P2M at leaves, M2M, multipole power */
    cplx *M = calloc((size_t)nc * nco, sizeof(cplx));
    cplx *F = calloc((size_t)nc * nco, sizeof(cplx));
    double *P = calloc((size_t)nc * (p + 1), sizeof(double));
    for (long ci = nc - 1; ci >= 0; --ci) { /* daughters always have larger indices */
        cell_t *c = &t->cells[ci];
        if (c->leaf) p2m(p, c->count, &t->xs[3 * c->first], &t->mus[c->first], c->s, &M[ci * nco]);
        else
            for (long j = 0; j < c->nchild; ++j)
                m2m(p, &M[(c->child + j) * nco], t->cells[c->child + j].s, c->s, &M[ci * nco]);
        multipole_power(p, &M[ci * nco], &P[ci * (p + 1)]);
    }

    /* dual tree walk */
    walk_t w = {0};
    w.t = t; w.p = p; w.mac = prm->mac; w.use_com = 0;
    w.adaptive = prm->adaptive_p && prm->mac != MAC_THETA;
    w.eps = prm->eps; w.theta_crit = prm->theta_crit;
    w.p2p_thresh = prm->p2p_c * pow((double)p, 3);
    w.P = P;
    walk(&w, 0, 0);
    run->m2l = w.m2l;
    run->p2p = w.p2p;
    run->st.n_m2l = w.m2l.n;
    run->st.n_p2p = w.p2p.n;

    /* interactions */
    for (long i = 0; i < w.m2l.n; ++i) {  /* each at its own order q <= p (F_n, n <= q; M_k, k <= q - n) */
        long A = w.m2l.v[i].a, B = w.m2l.v[i].b;
        m2l(w.m2l.v[i].q, &M[A * nco], t->cells[A].s, t->cells[B].s, &F[B * nco]);
    }
    double *ps = calloc(n, sizeof(double)), *ac = calloc(3 * n, sizeof(double));
    long coin = 0, inter = 0;
    for (long i = 0; i < w.p2p.n; ++i) {
        long A = w.p2p.v[i].a, B = w.p2p.v[i].b;
        p2p_pair(t, A, B, ps, ac, &coin, 0);
        inter += t->cells[A].count * t->cells[B].count - (A == B ? t->cells[A].count : 0);
    }
    double *tn = NULL;
    if (prm->want_tidal) {
        tn = calloc(6 * n, sizeof(double));
        for (long i = 0; i < w.p2p.n; ++i) p2p_tidal_pair(t, w.p2p.v[i].a, w.p2p.v[i].b, tn);
        free(run->tidal);
        run->tidal = calloc(6 * n, sizeof(double));
    }
    run->st.p2p_interactions = inter;
    run->st.coincident = coin;

    /* downward pass: L2L, then L2P at the leaves; daughters have larger indices */
    for (long ci = 0; ci < nc; ++ci) {
        cell_t *c = &t->cells[ci];
        if (!c->leaf) {
            for (long j = 0; j < c->nchild; ++j)
                l2l(p, &F[ci * nco], c->s, t->cells[c->child + j].s, &F[(c->child + j) * nco]);
        } else {
            for (long i = c->first; i < c->first + c->count; ++i) {
                long o = t->perm[i];
                if (!t->act[i]) {
                    run->psi[o] = NAN;
                    for (int d = 0; d < 3; ++d) run->acc[3 * o + d] = NAN;
                    if (tn) for (int d = 0; d < 6; ++d) run->tidal[6 * o + d] = NAN;
                    continue;
                }
                double psi_l, a[3], Tf[6];
                l2p_t(p, &F[ci * nco], c->s, &t->xs[3 * i], &psi_l, a, tn ? Tf : NULL);
                if (tn) for (int d = 0; d < 6; ++d) run->tidal[6 * o + d] = G * (Tf[d] + tn[6 * i + d]);
                run->psi[o] = G * (psi_l + ps[i]);
                for (int d = 0; d < 3; ++d) run->acc[3 * o + d] = G * (a[d] + ac[3 * i + d]);
            }
        }
    }
    free(ps); free(ac); free(M); free(F); free(P); free(tn);
}

/* Sec. 7.1's re-cycled tree: the particle order, cells and centres of the run prev (the same
 * n particles in the same caller order) for new positions x and masses mu; radii, masses
 * and centres of mass are recomputed, then the evaluation proceeds as usual */
orc_run *orc_fmm_reuse(const orc_run *prev, long n, const double *x, const double *mu, double G,
                       const orc_params *prm, const double *scale_in, const unsigned char *active,
                       const double *eps_b)
{
    if (!prev || prev->t.n != n || n <= 0 || !prm || prm->p < 1 || prm->p > 20) return NULL;
    if (prm->mac != MAC_THETA && !(prm->eps > 0)) return NULL;
    for (long i = 0; i < n; ++i) {
        if (!isfinite(x[3 * i]) || !isfinite(x[3 * i + 1]) || !isfinite(x[3 * i + 2]) ||
            !isfinite(mu[i]) || mu[i] < 0)
            return NULL;
    }
    orc_run *run = calloc(1, sizeof(orc_run));
    run->prm = *prm;
    run->psi = calloc(n, sizeof(double));
    run->acc = calloc(3 * n, sizeof(double));
    tree_t *t = &run->t;
    const tree_t *o = &prev->t;
    t->n = n;
    t->leaf_size = o->leaf_size;
    t->ncells = t->cap = o->ncells;
    for (int k = 0; k < 3; ++k) t->lo[k] = o->lo[k];
    t->side = o->side;
    t->cells = malloc(sizeof(cell_t) * o->ncells);
    memcpy(t->cells, o->cells, sizeof(cell_t) * o->ncells);
    t->perm = malloc(sizeof(long) * n);
    memcpy(t->perm, o->perm, sizeof(long) * n);
    t->keys = NULL;
    t->xs = malloc(sizeof(double) * 3 * n);
    t->mus = malloc(sizeof(double) * n);
    for (long i = 0; i < n; ++i) {
        const long j = t->perm[i];
        for (int k = 0; k < 3; ++k) t->xs[3 * i + k] = x[3 * j + k];
        t->mus[i] = mu[j];
    }
    cell_geometry_k(t, 0, 1);
    evaluate_on_tree(run, G, scale_in, active, eps_b);
    return run;
}

orc_run *orc_fmm(long n, const double *x, const double *mu, double G, const orc_params *prm,
                 const double *scale_in /* caller order, may be NULL */)
{
    return orc_fmm_active(n, x, mu, G, prm, scale_in, NULL, NULL);
}

void orc_run_free(orc_run *run)
{
    if (!run) return;
    free_tree(&run->t);
    free(run->m2l.v); free(run->p2p.v);
    free(run->scale_sorted); free(run->psi); free(run->acc); free(run->tidal);
    free(run);
}

/* accessors used by the Python test wrapper */
int orc_run_tidal(const orc_run *run, double *T)
{
    if (!run->tidal) return 0;
    memcpy(T, run->tidal, sizeof(double) * 6 * run->t.n);
    return 1;
}
void orc_run_outputs(const orc_run *run, double *psi, double *acc)
{
    memcpy(psi, run->psi, sizeof(double) * run->t.n);
    memcpy(acc, run->acc, sizeof(double) * 3 * run->t.n);
}
void orc_run_stats(const orc_run *run, orc_stats *st) { *st = run->st; }
long orc_run_ncells(const orc_run *run) { return run->t.ncells; }
/* per cell: level, leaf, first, count, nchild, then s[3], rho, mass, minscale */
void orc_run_cells(const orc_run *run, long *ints /* [nc][5] */, double *dbl /* [nc][6] */)
{
    for (long i = 0; i < run->t.ncells; ++i) {
        const cell_t *c = &run->t.cells[i];
        ints[5 * i] = c->level; ints[5 * i + 1] = c->leaf; ints[5 * i + 2] = c->first;
        ints[5 * i + 3] = c->count; ints[5 * i + 4] = c->nchild;
        dbl[6 * i] = c->s[0]; dbl[6 * i + 1] = c->s[1]; dbl[6 * i + 2] = c->s[2];
        dbl[6 * i + 3] = c->rho; dbl[6 * i + 4] = c->mass; dbl[6 * i + 5] = c->minscale;
    }
}
/* interaction lists as (source cell, sink cell) index pairs */
void orc_run_lists(const orc_run *run, long *m2l /* [n_m2l][2] */, long *p2p /* [n_p2p][2] */)
{
    for (long i = 0; i < run->m2l.n; ++i) { m2l[2 * i] = run->m2l.v[i].a; m2l[2 * i + 1] = run->m2l.v[i].b; }
    for (long i = 0; i < run->p2p.n; ++i) { p2p[2 * i] = run->p2p.v[i].a; p2p[2 * i + 1] = run->p2p.v[i].b; }
}
void orc_run_m2l_orders(const orc_run *run, int *q)
{
    for (long i = 0; i < run->m2l.n; ++i) q[i] = run->m2l.v[i].q;
}
/* The single-interaction experiment of Sec. 4 (its Figs. 2-3): the particles of sink cell B
 * receive the interaction of source cell A through the chain P2M (eq. 3c, about z_A = s_A),
 * M2L (eq. 3b, to s_B) and L2P (eqs. 3a, 7) at order p, and the FP64 direct sum of A's
 * particles (eq. 1) is the truth.  out[0] = max over b in B of delta a_b r^2 / M_A;
 * out[1] = max over b of delta a_b / |a_b|, a_b the true acceleration due to A;
 * out[2] = E~_{A->B} of eq. (17) (from orc_mac_lhs, times r^2 / M_A); out[3] = theta of
 * eq. (9) with rho_z = rho_s = rho.  Returns 0 when A or B is not a cell of the run, A has
 * no mass, or A = B. */
int orc_interaction_errors(const orc_run *run, long A, long B, int p, double *out)
{
    const tree_t *t = &run->t;
    if (A < 0 || B < 0 || A >= t->ncells || B >= t->ncells || A == B || p < 1 || p > 20) return 0;
    const cell_t *a = &t->cells[A], *b = &t->cells[B];
    if (!(a->mass > 0)) return 0;
    const int nco = NCOEF(p);
    cplx *M = calloc(nco, sizeof(cplx)), *F = calloc(nco, sizeof(cplx));
    double *P = calloc(p + 1, sizeof(double));
    p2m(p, a->count, &t->xs[3 * a->first], &t->mus[a->first], a->s, M);
    multipole_power(p, M, P);
    m2l(p, M, a->s, b->s, F);
    const double r = dist3(b->s, a->s);
    double e_abs = 0, e_rel = 0;
    for (long i = b->first; i < b->first + b->count; ++i) {
        const double *xb = &t->xs[3 * i];
        double psi_l, af[3], at[3] = {0, 0, 0};
        l2p(p, F, b->s, xb, &psi_l, af);
        for (long j = a->first; j < a->first + a->count; ++j) {
            const double d[3] = {t->xs[3 * j] - xb[0], t->xs[3 * j + 1] - xb[1], t->xs[3 * j + 2] - xb[2]};
            const double rr = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
            const double q = t->mus[j] / (rr * rr * rr);
            for (int k = 0; k < 3; ++k) at[k] += q * d[k];
        }
        const double da = sqrt((af[0] - at[0]) * (af[0] - at[0]) + (af[1] - at[1]) * (af[1] - at[1]) +
                               (af[2] - at[2]) * (af[2] - at[2]));
        const double an = sqrt(at[0] * at[0] + at[1] * at[1] + at[2] * at[2]);
        if (da * r * r / a->mass > e_abs) e_abs = da * r * r / a->mass;
        if (an > 0 && da / an > e_rel) e_rel = da / an;
    }
    out[0] = e_abs;
    out[1] = e_rel;
    out[2] = orc_mac_lhs(p, P, r, a->rho, b->rho) * r * r / a->mass;
    out[3] = (a->rho + b->rho) / r;
    free(M); free(F); free(P);
    return 1;
}
void orc_run_perm(const orc_run *run, long *perm) { memcpy(perm, run->t.perm, sizeof(long) * run->t.n); }
void orc_run_scale(const orc_run *run, double *scale_sorted)
{
    if (run->scale_sorted) memcpy(scale_sorted, run->scale_sorted, sizeof(double) * run->t.n);
}
