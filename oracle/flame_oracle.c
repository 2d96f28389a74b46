/*
 * flame_oracle.c -- plain FP64 CPU oracle of one FLAME lattice-Boltzmann
 * Hall-MHD time step (Foldes et al., "Efficient kinetic Lattice Boltzmann
 * simulation of three-dimensional Hall-MHD Turbulence", arXiv 2212.11024).
 *
 * TEST INFRASTRUCTURE.  Only the test suite, the package smoke check and the
 * benchmark's CPU-baseline leg may load this library.  It shares no code,
 * header, table or helper with the CUDA implementation.
 *
 * What it computes, per lattice site and time step, in the paper's order:
 *   1. rho, U from the fluid populations (Sec. 3.1.1, eq. LB_moments2);
 *      B and Lambda from the magnetic populations (Sec. 3.2, eqs.
 *      mag_field_LB and LB_density_current).
 *   2. J from the 3x3 linear system (Sec. 3.2, eqs. soe_current_density /
 *      soe_objects, App. B), solved by Gaussian elimination.
 *   3. f^mhd(0): the 6th-order Hermite equilibrium of App. A plus the
 *      Lorentz stress term (Sec. 3.1.1).
 *   4. Central-moment collision (Sec. 3.1.2, eqs. cm_collision_step and
 *      collision_matrix, App. A): k = T^T f, k* = k - S(k - k^eq),
 *      f* = (T^T)^-1 k*, with T(U) built per site and inverted by LU.
 *   5. Hall magnetic equilibrium (eq. gHall_eq) and BGK relaxation
 *      (eq. MHD_LBscheme).
 *   6. Streaming (eq. stream), periodic, by pulling into a second array.
 *
 * Readings of the paper taken here (each one is a correction of a printed
 * formula that the moment identities the paper states decide):
 *   - D3Q27 edge weight is 1/54 (Sec. 3.1.1); App. A prints 8/27.
 *   - The Lorentz term is w_i H2_i : (|B|^2 I/2 - BB) / (2 cs^4), the form
 *     whose second moment is the Maxwell stress the paper requires
 *     (eq. after the f^mhd(0) definition); the printed expression
 *     (|B|^2 |c|^2 - (c.B)^2) adds mass 3|B|^2 and is kept only as
 *     oracle_lorentz_printed() for the test that documents it.
 *   - Third-order basis vectors T11, T12, T14, T15 are garbled in print
 *     (the printed set is singular); the basis used is
 *     T10..T15 = xy^2+xz^2, x^2y+yz^2, x^2z+y^2z, xy^2-xz^2, x^2y-yz^2,
 *     x^2z-y^2z of cbar = c - U.
 *   - The Hermite terms of App. A with garbled subscripts are the terms in
 *     which every Cartesian index appears at most twice (the D3Q27 set).
 *   - Current: J = curl B = -(omega_B/C^2) eps_{g a b}(Lambda-Lambda0)_{ab},
 *     so the linear system is J + s J x B = y with s = 2 alpha_H omega_B/C^2
 *     and y = -(omega_B/C^2)(A - 2 U x B), A_g = eps_{g a b} Lambda_{ab}.
 *
 * Lattice units: dx = dt = 1, cs^2 = 1/3, C^2 = 1/4 (2C = sqrt(3) cs),
 * omega = 1/tau_nu, omega_B = 1/tau_eta, alpha_H = d_i.
 *
 * Population array layout: pop[q][z][y][x], x fastest; q = 0..26 fluid in
 * the App. A velocity order; q = 27 + 7*b + i magnetic component b (x,y,z)
 * on D3Q7 velocity i (rest, +x, -x, +y, -y, +z, -z).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define NQ 27
#define NM 7
#define NPOP 48

/* App. A: D3Q27 velocity set, in the order printed there. */
static const int CV[NQ][3] = {
    {0, 0, 0},    {-1, 0, 0},  {0, -1, 0},  {0, 0, -1},  {-1, -1, 0},
    {-1, 1, 0},   {-1, 0, -1}, {-1, 0, 1},  {0, -1, -1}, {0, -1, 1},
    {-1, -1, -1}, {-1, -1, 1}, {-1, 1, -1}, {-1, 1, 1},  {1, 0, 0},
    {0, 1, 0},    {0, 0, 1},   {1, 1, 0},   {1, -1, 0},  {1, 0, 1},
    {1, 0, -1},   {0, 1, 1},   {0, 1, -1},  {1, 1, 1},   {1, 1, -1},
    {1, -1, 1},   {1, -1, -1}};

/* Sec. 3.2: D3Q7 velocity set (rest and the six faces). */
static const int XV[NM][3] = {{0, 0, 0},  {1, 0, 0},  {-1, 0, 0}, {0, 1, 0},
                              {0, -1, 0}, {0, 0, 1},  {0, 0, -1}};

static const double CS2 = 1.0 / 3.0; /* Sec. 3.1.1: dx/dt = sqrt(3) cs */
static const double CC2 = 0.25;      /* eq. lattice_coincidence: 2C = sqrt(3) cs */

/* Sec. 3.1.1: w = 8/27, 2/27, 1/54, 1/216 for centre, face, edge, corner. */
static double w27(int i) {
    int n = CV[i][0] * CV[i][0] + CV[i][1] * CV[i][1] + CV[i][2] * CV[i][2];
    if (n == 0) return 8.0 / 27.0;
    if (n == 1) return 2.0 / 27.0;
    if (n == 2) return 1.0 / 54.0;
    return 1.0 / 216.0;
}

/* Sec. 3.2: W_centre = 1/4, W_face = 1/8. */
static double w7(int i) { return i == 0 ? 0.25 : 0.125; }

/* ------------------------------------------------------------------ */
/* Hermite tensors and the App. A equilibrium                          */
/* ------------------------------------------------------------------ */

/* H^(n)_{idx}(c) by the Hermite recurrence for a Gaussian of variance
 * cs^2:  H_{a,I} = c_a H_I - cs^2 sum_{j: I_j = a} H_{I without j}. */
static double hermite(const double c[3], const int *idx, int n) {
    if (n == 0) return 1.0;
    int a = idx[0];
    const int *rest = idx + 1;
    double h = c[a] * hermite(c, rest, n - 1);
    for (int j = 0; j < n - 1; ++j) {
        if (rest[j] != a) continue;
        int sub[8];
        int m = 0;
        for (int k = 0; k < n - 1; ++k)
            if (k != j) sub[m++] = rest[k];
        h -= CS2 * hermite(c, sub, n - 2);
    }
    return h;
}

/* The 27 terms of App. A: a term is (nx, ny, nz) copies of the indices
 * x, y, z, each at most twice; its prefactor is 1/(nx! ny! nz! cs^(2n)).
 * (That reproduces App. A: 1/(2cs^4) for xx, 2/(2cs^4) for xy, 1/(2cs^6)
 * for xxy, 2/(2cs^6) for xyz, 1/(4cs^8) for xxyy, 2/(4cs^8) for xyzz,
 * 1/(4cs^10) for xxyzz and 1/(8cs^12) for xxyyzz.) */
static int g_term_n[NQ][3];
static double g_term_coef[NQ];
static double g_hval[NQ][NQ]; /* [term][population] */
static int g_tables_ready = 0;

static void build_tables(void) {
    if (g_tables_ready) return;
    int t = 0;
    for (int nz = 0; nz <= 2; ++nz)
        for (int ny = 0; ny <= 2; ++ny)
            for (int nx = 0; nx <= 2; ++nx) {
                static const double fact[3] = {1.0, 1.0, 2.0};
                int n = nx + ny + nz;
                g_term_n[t][0] = nx;
                g_term_n[t][1] = ny;
                g_term_n[t][2] = nz;
                g_term_coef[t] = 1.0 / (fact[nx] * fact[ny] * fact[nz] * pow(CS2, n));
                int idx[8];
                int m = 0;
                for (int k = 0; k < nx; ++k) idx[m++] = 0;
                for (int k = 0; k < ny; ++k) idx[m++] = 1;
                for (int k = 0; k < nz; ++k) idx[m++] = 2;
                for (int i = 0; i < NQ; ++i) {
                    double c[3] = {CV[i][0], CV[i][1], CV[i][2]};
                    g_hval[t][i] = hermite(c, idx, n);
                }
                ++t;
            }
    g_tables_ready = 1;
}

/* App. A: f^(0)_i = w_i rho sum_terms coef * H_term(c_i) * U^term. */
void oracle_feq_hermite(double rho, const double U[3], double out[NQ]) {
    build_tables();
    double mono[NQ];
    for (int t = 0; t < NQ; ++t) {
        double m = 1.0;
        for (int a = 0; a < 3; ++a)
            for (int k = 0; k < g_term_n[t][a]; ++k) m *= U[a];
        mono[t] = g_term_coef[t] * m;
    }
    for (int i = 0; i < NQ; ++i) {
        double s = 0.0;
        for (int t = 0; t < NQ; ++t) s += g_hval[t][i] * mono[t];
        out[i] = w27(i) * rho * s;
    }
}

/* Closed form of the same sum: it factorises over the three axes into
 * rho * prod_a psi(c_a, U_a), psi(0,u) = 2/3 - u^2,
 * psi(+-1,u) = (1/3 + u^2 +- u)/2. */
void oracle_feq_product(double rho, const double U[3], double out[NQ]) {
    for (int i = 0; i < NQ; ++i) {
        double p = rho;
        for (int a = 0; a < 3; ++a) {
            double u = U[a];
            int c = CV[i][a];
            p *= (c == 0) ? (2.0 / 3.0 - u * u) : 0.5 * (1.0 / 3.0 + u * u + c * u);
        }
        out[i] = p;
    }
}

/* Sec. 3.1.1 Lorentz stress term, moment-matching form:
 * w_i/(2 cs^4) H2_i : M with M = |B|^2 I/2 - B B. */
void oracle_lorentz(const double B[3], double out[NQ]) {
    double M[3][3];
    double b2 = B[0] * B[0] + B[1] * B[1] + B[2] * B[2];
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) M[a][b] = (a == b ? 0.5 * b2 : 0.0) - B[a] * B[b];
    for (int i = 0; i < NQ; ++i) {
        double s = 0.0;
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) {
                double h2 = CV[i][a] * CV[i][b] - (a == b ? CS2 : 0.0);
                s += h2 * M[a][b];
            }
        out[i] = w27(i) / (2.0 * CS2 * CS2) * s;
    }
}

/* The Lorentz term exactly as printed in Sec. 3.1.1 / App. A. Not used by
 * the step; kept so that a test can show it does not conserve mass. */
void oracle_lorentz_printed(const double B[3], double out[NQ]) {
    double b2 = B[0] * B[0] + B[1] * B[1] + B[2] * B[2];
    for (int i = 0; i < NQ; ++i) {
        double c2 = CV[i][0] * CV[i][0] + CV[i][1] * CV[i][1] + CV[i][2] * CV[i][2];
        double cb = CV[i][0] * B[0] + CV[i][1] * B[1] + CV[i][2] * B[2];
        out[i] = w27(i) / (2.0 * CS2 * CS2) * (b2 * c2 - cb * cb);
    }
}

/* ------------------------------------------------------------------ */
/* Central-moment collision                                            */
/* ------------------------------------------------------------------ */

/* Sec. 3.1.2 / App. A: the 27 basis monomials T_j evaluated at cbar. */
static void cm_basis(const double cb[3], double T[NQ]) {
    double x = cb[0], y = cb[1], z = cb[2];
    double x2 = x * x, y2 = y * y, z2 = z * z;
    T[0] = 1.0;
    T[1] = x;
    T[2] = y;
    T[3] = z;
    T[4] = x * y;
    T[5] = x * z;
    T[6] = y * z;
    T[7] = x2 - y2;
    T[8] = x2 - z2;
    T[9] = x2 + y2 + z2;
    T[10] = x * y2 + x * z2;
    T[11] = x2 * y + y * z2;
    T[12] = x2 * z + y2 * z;
    T[13] = x * y2 - x * z2;
    T[14] = x2 * y - y * z2;
    T[15] = x2 * z - y2 * z;
    T[16] = x * y * z;
    T[17] = x2 * y2 + x2 * z2 + y2 * z2;
    T[18] = x2 * y2 + x2 * z2 - y2 * z2;
    T[19] = x2 * y2 - x2 * z2;
    T[20] = x2 * y * z;
    T[21] = x * y2 * z;
    T[22] = x * y * z2;
    T[23] = x * y2 * z2;
    T[24] = x2 * y * z2;
    T[25] = x2 * y2 * z;
    T[26] = x2 * y2 * z2;
}

/* T(U) as a row-major 27x27 matrix, T[i*27 + j] = T_j(c_i - U). */
void oracle_cm_matrix(const double U[3], double T[NQ * NQ]) {
    for (int i = 0; i < NQ; ++i) {
        double cb[3] = {CV[i][0] - U[0], CV[i][1] - U[1], CV[i][2] - U[2]};
        cm_basis(cb, T + i * NQ);
    }
}

/* Solve A x = b (n x n, row-major, destroyed) by Gaussian elimination with
 * partial pivoting.  Returns 0, or -1 if a pivot is exactly zero. */
static int gauss_solve(double *A, double *b, int n, double *x) {
    for (int k = 0; k < n; ++k) {
        int p = k;
        double best = fabs(A[k * n + k]);
        for (int r = k + 1; r < n; ++r) {
            double v = fabs(A[r * n + k]);
            if (v > best) {
                best = v;
                p = r;
            }
        }
        if (best == 0.0) return -1;
        if (p != k) {
            for (int c = 0; c < n; ++c) {
                double t = A[k * n + c];
                A[k * n + c] = A[p * n + c];
                A[p * n + c] = t;
            }
            double t = b[k];
            b[k] = b[p];
            b[p] = t;
        }
        for (int r = k + 1; r < n; ++r) {
            double m = A[r * n + k] / A[k * n + k];
            if (m == 0.0) continue;
            for (int c = k; c < n; ++c) A[r * n + c] -= m * A[k * n + c];
            b[r] -= m * b[k];
        }
    }
    for (int k = n - 1; k >= 0; --k) {
        double s = b[k];
        for (int c = k + 1; c < n; ++c) s -= A[k * n + c] * x[c];
        x[k] = s / A[k * n + k];
    }
    return 0;
}

/* eq. cm_collision_step: k = T^T f, k^eq = T^T f^eq, k* = k - S (k - k^eq),
 * f* = (T^T)^{-1} k*.  S is the diagonal of the collision matrix. */
int oracle_collide_cm_literal(const double f[NQ], const double feq[NQ], const double U[3],
                              const double S[NQ], double out[NQ]) {
    double T[NQ * NQ];
    oracle_cm_matrix(U, T);
    double A[NQ * NQ]; /* A = T^T : A[j][i] = T_j(cbar_i) */
    double k[NQ], keq[NQ], ks[NQ];
    for (int j = 0; j < NQ; ++j) {
        double s = 0.0, se = 0.0;
        for (int i = 0; i < NQ; ++i) {
            A[j * NQ + i] = T[i * NQ + j];
            s += T[i * NQ + j] * f[i];
            se += T[i * NQ + j] * feq[i];
        }
        k[j] = s;
        keq[j] = se;
    }
    for (int j = 0; j < NQ; ++j) ks[j] = k[j] - S[j] * (k[j] - keq[j]);
    return gauss_solve(A, ks, NQ, out);
}

/* Second mode, same result: central moments in the monomial basis
 * kappa_abc = sum_i f_i cbar_x^a cbar_y^b cbar_z^c (a,b,c <= 2), the
 * relaxation of eq. collision_matrix written in that basis (the five
 * deviatoric second-order moments relax with omega, the trace and every
 * other moment take their equilibrium value), and the exact inverse of
 * the monomial transform, which is a product of one-dimensional maps
 * from (m0, m1, m2) at shift u to the populations at c = 0, +1, -1:
 *   f_0 = m0 (1 - u^2) - 2 u m1 - m2,
 *   f_+-1 = (m0 (u^2 +- u) + m1 (2u +- 1) + m2) / 2.
 * Only valid for the collision matrix of eq. collision_matrix. */
static double mono1(double cb, int a) { return a == 0 ? 1.0 : (a == 1 ? cb : cb * cb); }

static double inv1(int c, double u, int a) {
    if (c == 0) return a == 0 ? 1.0 - u * u : (a == 1 ? -2.0 * u : -1.0);
    double s = (double)c;
    if (a == 0) return 0.5 * (u * u + s * u);
    if (a == 1) return 0.5 * (2.0 * u + s);
    return 0.5;
}

void oracle_collide_cm_factored(const double f[NQ], const double feq[NQ], const double U[3],
                                double omega, double out[NQ]) {
    double kap[3][3][3], keq[3][3][3];
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b)
            for (int c = 0; c < 3; ++c) {
                double s = 0.0, se = 0.0;
                for (int i = 0; i < NQ; ++i) {
                    double m = mono1(CV[i][0] - U[0], a) * mono1(CV[i][1] - U[1], b) *
                               mono1(CV[i][2] - U[2], c);
                    s += m * f[i];
                    se += m * feq[i];
                }
                kap[a][b][c] = s;
                keq[a][b][c] = se;
            }
    double ks[3][3][3];
    memcpy(ks, keq, sizeof(ks));
    double r = 1.0 - omega;
    ks[1][1][0] += r * (kap[1][1][0] - keq[1][1][0]);
    ks[1][0][1] += r * (kap[1][0][1] - keq[1][0][1]);
    ks[0][1][1] += r * (kap[0][1][1] - keq[0][1][1]);
    double dxx = kap[2][0][0] - keq[2][0][0];
    double dyy = kap[0][2][0] - keq[0][2][0];
    double dzz = kap[0][0][2] - keq[0][0][2];
    double tr = (dxx + dyy + dzz) / 3.0;
    ks[2][0][0] += r * (dxx - tr);
    ks[0][2][0] += r * (dyy - tr);
    ks[0][0][2] += r * (dzz - tr);
    for (int i = 0; i < NQ; ++i) {
        double s = 0.0;
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b)
                for (int c = 0; c < 3; ++c)
                    s += ks[a][b][c] * inv1(CV[i][0], U[0], a) * inv1(CV[i][1], U[1], b) *
                         inv1(CV[i][2], U[2], c);
        out[i] = s;
    }
}

/* ------------------------------------------------------------------ */
/* Magnetic part                                                       */
/* ------------------------------------------------------------------ */

/* Sec. 3.2, eqs. soe_current_density / soe_objects: solve
 * (I + s M) J = y,  M J = J x B,  s = 2 alpha_H omega_B / C^2,
 * y = -(omega_B / C^2) (A - 2 U x B),  A_x = Lam_yz - Lam_zy, ...
 * Lam[3a+b] = Lambda_ab.  literal=1: Gaussian elimination on the 3x3
 * matrix; literal=0: closed form (y - s y x B + s^2 (y.B) B)/(1+s^2|B|^2). */
int oracle_current(int literal, const double Lam[9], const double U[3], const double B[3],
                   double omegaB, double alphaH, double J[3]) {
    double A[3] = {Lam[1 * 3 + 2] - Lam[2 * 3 + 1], Lam[2 * 3 + 0] - Lam[0 * 3 + 2],
                   Lam[0 * 3 + 1] - Lam[1 * 3 + 0]};
    double uxb[3] = {U[1] * B[2] - U[2] * B[1], U[2] * B[0] - U[0] * B[2],
                     U[0] * B[1] - U[1] * B[0]};
    double g = omegaB / CC2;
    double s = 2.0 * alphaH * omegaB / CC2;
    double y[3];
    for (int a = 0; a < 3; ++a) y[a] = -g * (A[a] - 2.0 * uxb[a]);
    if (literal) {
        double Mt[9] = {1.0, s * B[2], -s * B[1], -s * B[2], 1.0, s * B[0],
                        s * B[1], -s * B[0], 1.0};
        return gauss_solve(Mt, y, 3, J);
    }
    double yxb[3] = {y[1] * B[2] - y[2] * B[1], y[2] * B[0] - y[0] * B[2],
                     y[0] * B[1] - y[1] * B[0]};
    double yb = y[0] * B[0] + y[1] * B[1] + y[2] * B[2];
    double b2 = B[0] * B[0] + B[1] * B[1] + B[2] * B[2];
    double den = 1.0 + s * s * b2;
    for (int a = 0; a < 3; ++a) J[a] = (y[a] - s * yxb[a] + s * s * yb * B[a]) / den;
    return 0;
}

/* eq. gHall_eq: g_{i b} = W_i (B_b + xi_{i a} (V_a B_b - B_a V_b) / C^2),
 * V = U - alpha_H J.  out[7*b + i]. */
void oracle_geq_hall(const double B[3], const double U[3], const double J[3], double alphaH,
                     double out[3 * NM]) {
    double V[3] = {U[0] - alphaH * J[0], U[1] - alphaH * J[1], U[2] - alphaH * J[2]};
    for (int b = 0; b < 3; ++b)
        for (int i = 0; i < NM; ++i) {
            double s = 0.0;
            for (int a = 0; a < 3; ++a) s += XV[i][a] * (V[a] * B[b] - B[a] * V[b]);
            out[b * NM + i] = w7(i) * (B[b] + s / CC2);
        }
}

/* ------------------------------------------------------------------ */
/* One site                                                            */
/* ------------------------------------------------------------------ */

static void site_moments(const double in[NPOP], double *rho, double U[3], double B[3],
                         double Lam[9]) {
    double r = 0.0, j[3] = {0.0, 0.0, 0.0};
    for (int i = 0; i < NQ; ++i) {
        r += in[i];
        for (int a = 0; a < 3; ++a) j[a] += in[i] * CV[i][a];
    }
    *rho = r;
    for (int a = 0; a < 3; ++a) U[a] = j[a] / r;
    for (int b = 0; b < 3; ++b) {
        double s = 0.0;
        for (int i = 0; i < NM; ++i) s += in[NQ + b * NM + i];
        B[b] = s;
        for (int a = 0; a < 3; ++a) {
            double l = 0.0;
            for (int i = 0; i < NM; ++i) l += XV[i][a] * in[NQ + b * NM + i];
            Lam[a * 3 + b] = l;
        }
    }
}

/* Collide one site: in[48] pre-collision populations -> out[48].
 * mom (may be NULL) receives rho, U[3], B[3], J[3], Tr(Lambda). */
int oracle_site_collide(const double in[NPOP], double tau_nu, double tau_eta, double d_i,
                        int literal, double out[NPOP], double *mom) {
    double omega = 1.0 / tau_nu, omegaB = 1.0 / tau_eta;
    double rho, U[3], B[3], Lam[9], J[3];
    site_moments(in, &rho, U, B, Lam);
    int rc = oracle_current(literal, Lam, U, B, omegaB, d_i, J);
    double feq[NQ], lor[NQ];
    if (literal)
        oracle_feq_hermite(rho, U, feq);
    else
        oracle_feq_product(rho, U, feq);
    oracle_lorentz(B, lor);
    for (int i = 0; i < NQ; ++i) feq[i] += lor[i];
    if (literal) {
        double S[NQ];
        for (int j = 0; j < NQ; ++j) S[j] = (j >= 4 && j <= 8) ? omega : 1.0;
        rc |= oracle_collide_cm_literal(in, feq, U, S, out);
    } else {
        oracle_collide_cm_factored(in, feq, U, omega, out);
    }
    double geq[3 * NM];
    oracle_geq_hall(B, U, J, d_i, geq);
    for (int q = 0; q < 3 * NM; ++q) out[NQ + q] = in[NQ + q] - omegaB * (in[NQ + q] - geq[q]);
    if (mom) {
        mom[0] = rho;
        for (int a = 0; a < 3; ++a) {
            mom[1 + a] = U[a];
            mom[4 + a] = B[a];
            mom[7 + a] = J[a];
        }
        mom[10] = Lam[0] + Lam[4] + Lam[8];
    }
    return rc;
}

/* Scheme variants (not the paper's default scheme):
 *   1  BGK fluid collision f* = f - omega (f - f^mhd(0)) (Sec. 3.1.1, eq.
 *      collision; the central-moment operator with S = omega I);
 *   2  electron MHD: U neglected against alpha_H J in the magnetic
 *      equilibrium (the extension named at the end of Sec. 5), i.e. V =
 *      -alpha_H J and the current system with U = 0;
 *   3  current from a finite-difference stencil: J = periodic central-
 *      difference curl of the pre-collision B field (Jfd, supplied by the
 *      caller), used in the Hall equilibrium instead of the 3x3 solve.
 * Variant 0 is oracle_site_collide. */
int oracle_site_collide_variant(const double in[NPOP], double tau_nu, double tau_eta, double d_i,
                                int literal, int variant, const double Jfd[3], double out[NPOP]) {
    double omega = 1.0 / tau_nu, omegaB = 1.0 / tau_eta;
    double rho, U[3], B[3], Lam[9], J[3];
    const double zero[3] = {0.0, 0.0, 0.0};
    site_moments(in, &rho, U, B, Lam);
    int rc = 0;
    if (variant == 3) {
        for (int a = 0; a < 3; ++a) J[a] = Jfd[a];
    } else {
        rc = oracle_current(literal, Lam, variant == 2 ? zero : U, B, omegaB, d_i, J);
    }
    double feq[NQ], lor[NQ];
    if (literal)
        oracle_feq_hermite(rho, U, feq);
    else
        oracle_feq_product(rho, U, feq);
    oracle_lorentz(B, lor);
    for (int i = 0; i < NQ; ++i) feq[i] += lor[i];
    if (variant == 1) {
        for (int i = 0; i < NQ; ++i) out[i] = in[i] - omega * (in[i] - feq[i]);
    } else if (literal) {
        double S[NQ];
        for (int j = 0; j < NQ; ++j) S[j] = (j >= 4 && j <= 8) ? omega : 1.0;
        rc |= oracle_collide_cm_literal(in, feq, U, S, out);
    } else {
        oracle_collide_cm_factored(in, feq, U, omega, out);
    }
    double geq[3 * NM];
    oracle_geq_hall(B, variant == 2 ? zero : U, J, d_i, geq);
    for (int q = 0; q < 3 * NM; ++q) out[NQ + q] = in[NQ + q] - omegaB * (in[NQ + q] - geq[q]);
    return rc;
}

/* ------------------------------------------------------------------ */
/* Grid-level driver                                                   */
/* ------------------------------------------------------------------ */

static inline long site_index(int x, int y, int z, int nx, int ny) {
    return ((long)z * ny + y) * nx + x;
}

static inline int wrap(int v, int n) {
    v %= n;
    return v < 0 ? v + n : v;
}

static int pop_velocity(int q, int c[3]) {
    if (q < NQ) {
        c[0] = CV[q][0];
        c[1] = CV[q][1];
        c[2] = CV[q][2];
    } else {
        int i = (q - NQ) % NM;
        c[0] = XV[i][0];
        c[1] = XV[i][1];
        c[2] = XV[i][2];
    }
    return 0;
}

/* Advance nsteps: collide every site into post[], then stream by pulling
 * pop(x, q) = post(x - c_q, q).  Returns the number of sites at which the
 * LU solve met a zero pivot (0 normally). */
long oracle_step(int nx, int ny, int nz, double tau_nu, double tau_eta, double d_i, int literal,
                 int nsteps, double *pop, double *post) {
    build_tables();
    long n3 = (long)nx * ny * nz;
    long bad = 0;
    for (int step = 0; step < nsteps; ++step) {
#pragma omp parallel for schedule(static) reduction(+ : bad)
        for (long s = 0; s < n3; ++s) {
            double in[NPOP], out[NPOP];
            for (int q = 0; q < NPOP; ++q) in[q] = pop[q * n3 + s];
            if (oracle_site_collide(in, tau_nu, tau_eta, d_i, literal, out, NULL) != 0) ++bad;
            for (int q = 0; q < NPOP; ++q) post[q * n3 + s] = out[q];
        }
#pragma omp parallel for schedule(static)
        for (long s = 0; s < n3; ++s) {
            int x = (int)(s % nx), y = (int)((s / nx) % ny), z = (int)(s / ((long)nx * ny));
            for (int q = 0; q < NPOP; ++q) {
                int c[3];
                pop_velocity(q, c);
                long src = site_index(wrap(x - c[0], nx), wrap(y - c[1], ny), wrap(z - c[2], nz),
                                      nx, ny);
                pop[q * n3 + s] = post[q * n3 + src];
            }
        }
    }
    return bad;
}

/* Second-order central difference, periodic:  d_a F at site s. */
static double cdiff(const double *F, int a, int x, int y, int z, int nx, int ny, int nz) {
    int p[3] = {x, y, z}, m[3] = {x, y, z};
    int n[3] = {nx, ny, nz};
    p[a] = wrap(p[a] + 1, n[a]);
    m[a] = wrap(m[a] - 1, n[a]);
    return 0.5 * (F[site_index(p[0], p[1], p[2], nx, ny)] - F[site_index(m[0], m[1], m[2], nx, ny)]);
}

/* oracle_step for a scheme variant (see oracle_site_collide_variant).  For
 * variant 3, B is computed at every site first and J = curl B by periodic
 * central differences.  `bfield` (3 N3 doubles) is scratch, may be NULL for
 * the other variants. */
long oracle_step_variant(int nx, int ny, int nz, double tau_nu, double tau_eta, double d_i, int literal,
                         int variant, int nsteps, double *pop, double *post, double *bfield) {
    build_tables();
    long n3 = (long)nx * ny * nz;
    long bad = 0;
    for (int step = 0; step < nsteps; ++step) {
        if (variant == 3) {
#pragma omp parallel for schedule(static)
            for (long s = 0; s < n3; ++s)
                for (int b = 0; b < 3; ++b) {
                    double v = 0.0;
                    for (int i = 0; i < NM; ++i) v += pop[(NQ + b * NM + i) * n3 + s];
                    bfield[b * n3 + s] = v;
                }
        }
#pragma omp parallel for schedule(static) reduction(+ : bad)
        for (long s = 0; s < n3; ++s) {
            double in[NPOP], out[NPOP], J[3] = {0.0, 0.0, 0.0};
            for (int q = 0; q < NPOP; ++q) in[q] = pop[q * n3 + s];
            if (variant == 3) {
                int x = (int)(s % nx), y = (int)((s / nx) % ny), z = (int)(s / ((long)nx * ny));
                double d[3][3];
                for (int a = 0; a < 3; ++a)
                    for (int b = 0; b < 3; ++b) d[a][b] = cdiff(bfield + b * n3, a, x, y, z, nx, ny, nz);
                J[0] = d[1][2] - d[2][1];
                J[1] = d[2][0] - d[0][2];
                J[2] = d[0][1] - d[1][0];
            }
            if (oracle_site_collide_variant(in, tau_nu, tau_eta, d_i, literal, variant, J, out) != 0) ++bad;
            for (int q = 0; q < NPOP; ++q) post[q * n3 + s] = out[q];
        }
#pragma omp parallel for schedule(static)
        for (long s = 0; s < n3; ++s) {
            int x = (int)(s % nx), y = (int)((s / nx) % ny), z = (int)(s / ((long)nx * ny));
            for (int q = 0; q < NPOP; ++q) {
                int c[3];
                pop_velocity(q, c);
                long src = site_index(wrap(x - c[0], nx), wrap(y - c[1], ny), wrap(z - c[2], nz),
                                      nx, ny);
                pop[q * n3 + s] = post[q * n3 + src];
            }
        }
    }
    return bad;
}

/* Initial populations from macroscopic fields (the paper only states the
 * fields; the populations are its equilibria plus first-order
 * non-equilibrium parts):
 *   f = f^(0)(rho,u) + Lorentz(B) + noneq * w_i H2_i : Pi^neq / (2 cs^4),
 *       Pi^neq = -(rho cs^2 / omega)(grad u + grad u^T);
 *   g = g^Hall(0)(u, B, J0) - noneq * (W_i / omega_B) xi_{i a} d_a B_b,
 *       J0 = curl B.
 * Fields are [comp][z][y][x]; rho may be NULL (rho = 1).  gradu / gradB
 * ([3a+b][z][y][x] = d_a F_b) may be NULL: periodic central differences. */
int oracle_init(int nx, int ny, int nz, double tau_nu, double tau_eta, double d_i,
                const double *rho_f, const double *u, const double *B, const double *gradu,
                const double *gradB, int noneq, double *pop) {
    build_tables();
    long n3 = (long)nx * ny * nz;
    double omega = 1.0 / tau_nu, omegaB = 1.0 / tau_eta;
#pragma omp parallel for schedule(static)
    for (long s = 0; s < n3; ++s) {
        int x = (int)(s % nx), y = (int)((s / nx) % ny), z = (int)(s / ((long)nx * ny));
        double rho = rho_f ? rho_f[s] : 1.0;
        double U[3] = {u[s], u[n3 + s], u[2 * n3 + s]};
        double Bv[3] = {B[s], B[n3 + s], B[2 * n3 + s]};
        double du[9], dB[9];
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) {
                du[3 * a + b] = gradu ? gradu[(3 * a + b) * n3 + s]
                                      : cdiff(u + b * n3, a, x, y, z, nx, ny, nz);
                dB[3 * a + b] = gradB ? gradB[(3 * a + b) * n3 + s]
                                      : cdiff(B + b * n3, a, x, y, z, nx, ny, nz);
            }
        double J0[3] = {dB[3 * 1 + 2] - dB[3 * 2 + 1], dB[3 * 2 + 0] - dB[3 * 0 + 2],
                        dB[3 * 0 + 1] - dB[3 * 1 + 0]};
        double feq[NQ], lor[NQ];
        oracle_feq_hermite(rho, U, feq);
        oracle_lorentz(Bv, lor);
        double Pi[3][3];
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b)
                Pi[a][b] = -(rho * CS2 / omega) * (du[3 * a + b] + du[3 * b + a]);
        for (int i = 0; i < NQ; ++i) {
            double ne = 0.0;
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b)
                    ne += (CV[i][a] * CV[i][b] - (a == b ? CS2 : 0.0)) * Pi[a][b];
            ne *= w27(i) / (2.0 * CS2 * CS2);
            pop[i * n3 + s] = feq[i] + lor[i] + (noneq ? ne : 0.0);
        }
        double geq[3 * NM];
        oracle_geq_hall(Bv, U, J0, d_i, geq);
        for (int b = 0; b < 3; ++b)
            for (int i = 0; i < NM; ++i) {
                double ne = 0.0;
                for (int a = 0; a < 3; ++a) ne += XV[i][a] * dB[3 * a + b];
                ne *= -w7(i) / omegaB;
                pop[(NQ + b * NM + i) * n3 + s] = geq[b * NM + i] + (noneq ? ne : 0.0);
            }
    }
    return 0;
}

/* Macroscopic fields of the pre-collision populations: rho [N3], u [3][N3],
 * B [3][N3], J [3][N3] (literal 3x3 solve), trlam [N3] = Tr(Lambda).
 * Any output may be NULL. */
void oracle_moments(int nx, int ny, int nz, double tau_eta, double d_i, const double *pop,
                    double *rho_o, double *u_o, double *B_o, double *J_o, double *trlam_o) {
    long n3 = (long)nx * ny * nz;
    double omegaB = 1.0 / tau_eta;
#pragma omp parallel for schedule(static)
    for (long s = 0; s < n3; ++s) {
        double in[NPOP];
        for (int q = 0; q < NPOP; ++q) in[q] = pop[q * n3 + s];
        double rho, U[3], Bv[3], Lam[9], J[3];
        site_moments(in, &rho, U, Bv, Lam);
        oracle_current(1, Lam, U, Bv, omegaB, d_i, J);
        if (rho_o) rho_o[s] = rho;
        for (int a = 0; a < 3; ++a) {
            if (u_o) u_o[a * n3 + s] = U[a];
            if (B_o) B_o[a * n3 + s] = Bv[a];
            if (J_o) J_o[a * n3 + s] = J[a];
        }
        if (trlam_o) trlam_o[s] = Lam[0] + Lam[4] + Lam[8];
    }
}

/* Lattice tables, for the tests that check them against the paper. */
void oracle_lattice(int c27[NQ * 3], double w[NQ], int xi7[NM * 3], double W[NM]) {
    for (int i = 0; i < NQ; ++i) {
        for (int a = 0; a < 3; ++a) c27[i * 3 + a] = CV[i][a];
        w[i] = w27(i);
    }
    for (int i = 0; i < NM; ++i) {
        for (int a = 0; a < 3; ++a) xi7[i * 3 + a] = XV[i][a];
        W[i] = w7(i);
    }
}

int oracle_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}
