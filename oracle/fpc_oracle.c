/*
 * fpc_oracle.c -- plain FP64 CPU oracle for the Fokker-Planck central-moment lattice Boltzmann
 * method for thermal convection (Schupbach & Premnath, arXiv 2504.09041).
 *
 * TEST INFRASTRUCTURE, NOT PRODUCT CODE.  This file is the slow, obviously-correct restatement of
 * the paper against which the CUDA path is checked.  Only the tests, the smoke check and the
 * benchmark's CPU-baseline leg may load it.  The product library never links, loads or calls it,
 * and the two share no code, tables or headers.
 *
 * Every per-node function follows the paper's steps in the paper's order and notation:
 *   - D2Q9 flow collision .......... Appendix A, Steps 1-5 (Step 7 for rho, u)
 *   - D2Q9 energy collision ........ Appendix B, Steps 1-5
 *   - D3Q15 energy collision ....... Appendix C, Steps 1-5
 *   - D3Q27 flow collision ......... Sec. 5.1-5.2 (moment definitions, attractors, Eq. forcing:3D);
 *                                    the full algorithm is deferred by the paper to its earlier work,
 *                                    so the reading used here is stated at orc_d3q27_collide.
 *   - streaming and walls .......... Eqs. LBMsteps-stream / LBMsteps-streamg, Sec. 6.1 (half-way
 *                                    bounce-back, anti-bounce-back), Boussinesq force Sec. 6.1 / 6.2
 *   - wall Nusselt number .......... Sec. 6.1 (second-order one-sided Lagrange derivative)
 *
 * Readings of garbled or silent passages (each also checked by a test):
 *   R1  App. A Step 2, kappa_22: the term printed "u_x^2 2 u_y kappa'_01" is -2 u_x^2 u_y kappa'_01.
 *   R2  App. B Step 2, eta_12: the printed kappa'_11 is eta'_11.
 *   R3  App. C Step 3 / Sec. 5.4: eta^Mv_012 = (2/3) c_s^2-hat eta~_010 (the factor c_s^2-hat is
 *       dropped once in Sec. 5.4 and present in App. C and in the recurrence).
 *   R4  Sec. 5.2 discrete kappa^Mv_122: the product "kappa~_011 kappa~_012" is kappa~_110 kappa~_012
 *       (continuous form of the same attractor and the recurrence Eq. Mvcmattractor3D).
 *   R5  Second-order sources are zero (Eq. sourceCM2D states sigma_20 = sigma_02 = sigma_11 = 0);
 *       higher-order sources use the pre-collision central moments.
 *   R6  D3Q27 flow: raw basis = the 27 tensor monomials; second-order diagonal moments relax as a
 *       trace (bulk rate) and two deviators (shear rate), by analogy with App. A Step 3; the cascade
 *       runs by order 0-3, 4, 5, 6, each attractor using the post-collision lower moments.
 *   R7  Walls cut half-way between nodes; a link whose source lies beyond a fixed-temperature face
 *       takes anti-bounce-back with that face's temperature, one beyond an adiabatic face
 *       bounce-back.  A link that crosses two or three walls (box edges and corners) takes the rule
 *       of the crossed face that comes last in the order -z, -y, -x, +x, +y, +z.  Periodic axes
 *       wrap first.
 *   R8  Eq. sourceCM2D prints sigma_12 = (F_x/rho) kappa_02 + (F_y/rho) kappa_11; the general
 *       source Eq. forcing:2D (factor n = 2 on the kappa_11 term) and the mirror term of sigma_21
 *       give sigma_12 = (F_x/rho) kappa_02 + 2 (F_y/rho) kappa_11, which is used here.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_PERIODIC 0
#define ORC_WALL_ADIABATIC 1
#define ORC_WALL_FIXED_T 2

/* c_s^2 = 1/3 (App. A Step 3) and c_s^2-hat = 1/3 (App. B Step 3). */
static const double CS2 = 1.0 / 3.0;
static const double CHS2 = 1.0 / 3.0;

/* ------------------------------------------------------------------------------------------ */
/* Velocity sets in the paper's order                                                          */
/* ------------------------------------------------------------------------------------------ */

/* D2Q9, Eqs. ex, ey. */
static const int D2Q9_E[9][3] = {
    {0, 0, 0}, {1, 0, 0}, {0, 1, 0}, {-1, 0, 0}, {0, -1, 0},
    {1, 1, 0}, {-1, 1, 0}, {-1, -1, 0}, {1, -1, 0}};

/* D3Q27, Sec. 5.2 (Cartesian components of the 27 links). */
static const int D3Q27_E[27][3] = {
    {0, 0, 0},   {1, 0, 0},   {-1, 0, 0},  {0, 1, 0},   {0, -1, 0},  {0, 0, 1},   {0, 0, -1},
    {1, 1, 0},   {-1, 1, 0},  {1, -1, 0},  {-1, -1, 0}, {1, 0, 1},   {-1, 0, 1},  {1, 0, -1},
    {-1, 0, -1}, {0, 1, 1},   {0, -1, 1},  {0, 1, -1},  {0, -1, -1}, {1, 1, 1},   {-1, 1, 1},
    {1, -1, 1},  {-1, -1, 1}, {1, 1, -1},  {-1, 1, -1}, {1, -1, -1}, {-1, -1, -1}};

/* D3Q15, Sec. 5.4. */
static const int D3Q15_E[15][3] = {
    {0, 0, 0},  {1, 0, 0},  {-1, 0, 0},  {0, 1, 0},  {0, -1, 0},
    {0, 0, 1},  {0, 0, -1}, {1, 1, 1},   {-1, 1, 1}, {1, -1, 1},
    {-1, -1, 1}, {1, 1, -1}, {-1, 1, -1}, {1, -1, -1}, {-1, -1, -1}};

/* D3Q27 central-moment order of Sec. 5.2: exponents (m, n, p) of each entry of m^c. */
static const int M27[27][3] = {
    {0, 0, 0}, {1, 0, 0}, {0, 1, 0}, {0, 0, 1}, {1, 1, 0}, {1, 0, 1}, {0, 1, 1},
    {2, 0, 0}, {0, 2, 0}, {0, 0, 2}, {1, 2, 0}, {1, 0, 2}, {2, 1, 0}, {0, 1, 2},
    {2, 0, 1}, {0, 2, 1}, {1, 1, 1}, {2, 2, 0}, {2, 0, 2}, {0, 2, 2}, {2, 1, 1},
    {1, 2, 1}, {1, 1, 2}, {1, 2, 2}, {2, 1, 2}, {2, 2, 1}, {2, 2, 2}};

enum {
    K000, K100, K010, K001, K110, K101, K011, K200, K020, K002, K120, K102, K210, K012,
    K201, K021, K111, K220, K202, K022, K211, K121, K112, K122, K212, K221, K222
};

static int k27_index(int m, int n, int p)
{
    for (int j = 0; j < 27; ++j)
        if (M27[j][0] == m && M27[j][1] == n && M27[j][2] == p) return j;
    return -1;
}

static double ipow(double x, int k)
{
    double r = 1.0;
    for (int i = 0; i < k; ++i) r *= x;
    return r;
}

static double binom(int n, int k)
{
    static const double t[3][3] = {{1, 0, 0}, {1, 1, 0}, {1, 2, 1}};
    return t[n][k];
}

/* ------------------------------------------------------------------------------------------ */
/* Appendix A / B, Steps 1, 2, 4, 5 on D2Q9 (identical for f and g).                           */
/* Moment order (00, 10, 01, 20, 02, 11, 21, 12, 22), Sec. 4.2.                                 */
/* ------------------------------------------------------------------------------------------ */

/* Step 1: raw moments m = P f. */
void orc_d2q9_step1(const double f[9], double r[9])
{
    r[0] = f[0] + f[1] + f[2] + f[3] + f[4] + f[5] + f[6] + f[7] + f[8];
    r[1] = f[1] - f[3] + f[5] - f[6] - f[7] + f[8];
    r[2] = f[2] - f[4] + f[5] + f[6] - f[7] - f[8];
    r[3] = f[1] + f[3] + f[5] + f[6] + f[7] + f[8];
    r[4] = f[2] + f[4] + f[5] + f[6] + f[7] + f[8];
    r[5] = f[5] - f[6] + f[7] - f[8];
    r[6] = f[5] + f[6] - f[7] - f[8];
    r[7] = f[5] - f[6] - f[7] + f[8];
    r[8] = f[5] + f[6] + f[7] + f[8];
}

/* Step 2: central moments m^c = F m (readings R1, R2). */
void orc_d2q9_step2(const double r[9], double ux, double uy, double c[9])
{
    const double uxx = ux * ux, uyy = uy * uy;
    c[0] = r[0];
    c[1] = r[1] - ux * r[0];
    c[2] = r[2] - uy * r[0];
    c[3] = r[3] - 2.0 * ux * r[1] + uxx * r[0];
    c[4] = r[4] - 2.0 * uy * r[2] + uyy * r[0];
    c[5] = r[5] - uy * r[1] - ux * r[2] + ux * uy * r[0];
    c[6] = r[6] - 2.0 * ux * r[5] + uxx * r[2] - uy * r[3] + 2.0 * ux * uy * r[1] - uxx * uy * r[0];
    c[7] = r[7] - 2.0 * uy * r[5] + uyy * r[1] - ux * r[4] + 2.0 * ux * uy * r[2] - ux * uyy * r[0];
    c[8] = r[8] - 2.0 * ux * r[7] + uxx * r[4] - 2.0 * uy * r[6] + 4.0 * ux * uy * r[5]
         - 2.0 * uxx * uy * r[2] + uyy * r[3] - 2.0 * ux * uyy * r[1] + uxx * uyy * r[0];
}

/* Step 4: raw moments from central moments, m = F^-1 m^c. */
void orc_d2q9_step4(const double c[9], double ux, double uy, double r[9])
{
    const double uxx = ux * ux, uyy = uy * uy;
    r[0] = c[0];
    r[1] = c[1] + ux * c[0];
    r[2] = c[2] + uy * c[0];
    r[3] = c[3] + 2.0 * ux * c[1] + uxx * c[0];
    r[4] = c[4] + 2.0 * uy * c[2] + uyy * c[0];
    r[5] = c[5] + ux * c[2] + uy * c[1] + ux * uy * c[0];
    r[6] = c[6] + 2.0 * ux * c[5] + uy * c[3] + uxx * c[2] + 2.0 * ux * uy * c[1] + uxx * uy * c[0];
    r[7] = c[7] + 2.0 * uy * c[5] + ux * c[4] + 2.0 * ux * uy * c[2] + uyy * c[1] + ux * uyy * c[0];
    r[8] = c[8] + 2.0 * ux * c[7] + 2.0 * uy * c[6] + 4.0 * ux * uy * c[5] + uyy * c[3]
         + uxx * c[4] + 2.0 * uxx * uy * c[2] + 2.0 * ux * uyy * c[1] + uxx * uyy * c[0];
}

/* Step 5: populations from raw moments, f = P^-1 m. */
void orc_d2q9_step5(const double r[9], double f[9])
{
    f[0] = r[0] - r[3] - r[4] + r[8];
    f[1] = (r[1] + r[3] - r[7] - r[8]) / 2.0;
    f[2] = (r[2] + r[4] - r[6] - r[8]) / 2.0;
    f[3] = (-r[1] + r[3] + r[7] - r[8]) / 2.0;
    f[4] = (-r[2] + r[4] + r[6] - r[8]) / 2.0;
    f[5] = (r[5] + r[6] + r[7] + r[8]) / 4.0;
    f[6] = (-r[5] + r[6] - r[7] + r[8]) / 4.0;
    f[7] = (r[5] - r[6] - r[7] + r[8]) / 4.0;
    f[8] = (-r[5] - r[6] + r[7] + r[8]) / 4.0;
}

/* Appendix A, Step 7: rho = sum f, rho u = sum f e + F/2. */
void orc_d2q9_macro(const double f[9], double Fx, double Fy, double out[3])
{
    double rho = 0.0, jx = 0.0, jy = 0.0;
    for (int a = 0; a < 9; ++a) {
        rho += f[a];
        jx += f[a] * D2Q9_E[a][0];
        jy += f[a] * D2Q9_E[a][1];
    }
    out[0] = rho;
    out[1] = (jx + 0.5 * Fx) / rho;
    out[2] = (jy + 0.5 * Fy) / rho;
}

/*
 * Appendix A, Steps 1-5: collision of the flow populations with the Boussinesq source.
 * om[0..8] are the paper's omega_0..omega_8 (omega_3 bulk on kappa_2s, omega_4 on kappa_2d,
 * omega_5 on kappa_11).  Sources follow Eq. sourceCM2D (reading R5), delta_t = 1.
 */
void orc_d2q9_f_collide(const double f[9], double rho, double ux, double uy, double Fx,
                        double Fy, const double om[9], double ft[9])
{
    double r[9], k[9], kt[9], rt[9];
    orc_d2q9_step1(f, r);
    orc_d2q9_step2(r, ux, uy, k);

    /* Step 3. */
    const double k2s = k[3] + k[4], k2d = k[3] - k[4];
    const double Mv00 = rho, Mv10 = 0.0, Mv01 = 0.0, Mv20 = CS2 * rho, Mv02 = CS2 * rho;
    const double Mv11 = 0.0, Mv21 = 0.0, Mv12 = 0.0;
    const double Mv2s = Mv20 + Mv02, Mv2d = Mv20 - Mv02;
    const double s00 = 0.0, s10 = Fx, s01 = Fy, s20 = 0.0, s02 = 0.0, s11 = 0.0;
    const double s2s = s20 + s02, s2d = s20 - s02;
    const double s21 = 2.0 * (Fx / rho) * k[5] + (Fy / rho) * k[3];
    const double s12 = (Fx / rho) * k[4] + 2.0 * (Fy / rho) * k[5]; /* reading R8 */
    const double s22 = 2.0 * ((Fx / rho) * k[7] + (Fy / rho) * k[6]);

    kt[0] = k[0] + om[0] * (Mv00 - k[0]) + (1.0 - om[0] / 2.0) * s00;
    kt[1] = k[1] + om[1] * (Mv10 - k[1]) + (1.0 - om[1] / 2.0) * s10;
    kt[2] = k[2] + om[2] * (Mv01 - k[2]) + (1.0 - om[2] / 2.0) * s01;
    const double kt2s = k2s + om[3] * (Mv2s - k2s) + (1.0 - om[3] / 2.0) * s2s;
    const double kt2d = k2d + om[4] * (Mv2d - k2d) + (1.0 - om[4] / 2.0) * s2d;
    kt[5] = k[5] + om[5] * (Mv11 - k[5]) + (1.0 - om[5] / 2.0) * s11;
    kt[6] = k[6] + om[6] * (Mv21 - k[6]) + (1.0 - om[6] / 2.0) * s21;
    kt[7] = k[7] + om[7] * (Mv12 - k[7]) + (1.0 - om[7] / 2.0) * s12;
    kt[3] = 0.5 * (kt2s + kt2d);
    kt[4] = 0.5 * (kt2s - kt2d);
    const double Mv22 = (kt[3] * kt[4] + 2.0 * kt[5] * kt[5]) / rho;
    kt[8] = k[8] + om[8] * (Mv22 - k[8]) + (1.0 - om[8] / 2.0) * s22;

    orc_d2q9_step4(kt, ux, uy, rt);
    orc_d2q9_step5(rt, ft);
}

/*
 * Appendix B, Steps 1-5: collision of the energy populations.  om[0..8] are the paper's
 * omega_0..omega_8 (omega_1 = omega_2 set by alpha).  The second-order pair is relaxed as
 * eta_2s = eta_20 + eta_02 and eta_2d = eta_20 - eta_02 with omega_3, omega_4 and then split
 * back, as in Appendix A.  option 0 takes the option-A attractors of orders 3-4 (Eq. MvT2D),
 * option 1 the renormalized option-B attractors (Eq. MvT2DoptionB), both from the
 * post-collision lower moments.
 */
void orc_d2q9_g_collide(const double g[9], double ux, double uy, const double om[9], int option,
                        double gt[9])
{
    double r[9], n[9], nt[9], rt[9];
    orc_d2q9_step1(g, r);
    orc_d2q9_step2(r, ux, uy, n);

    const double T = n[0];
    const double Mv00 = T, Mv10 = 0.0, Mv01 = 0.0, Mv20 = CHS2 * T, Mv02 = CHS2 * T, Mv11 = 0.0;
    const double n2s = n[3] + n[4], n2d = n[3] - n[4];
    const double Mv2s = Mv20 + Mv02, Mv2d = Mv20 - Mv02;

    nt[0] = n[0] + om[0] * (Mv00 - n[0]);
    nt[1] = n[1] + om[1] * (Mv10 - n[1]);
    nt[2] = n[2] + om[2] * (Mv01 - n[2]);
    const double nt2s = n2s + om[3] * (Mv2s - n2s);
    const double nt2d = n2d + om[4] * (Mv2d - n2d);
    nt[5] = n[5] + om[5] * (Mv11 - n[5]);
    nt[3] = 0.5 * (nt2s + nt2d);
    nt[4] = 0.5 * (nt2s - nt2d);

    double Mv21, Mv12, Mv22;
    if (option == 0) {
        Mv21 = (2.0 / 3.0) * CHS2 * nt[2];
        Mv12 = (2.0 / 3.0) * CHS2 * nt[1];
        Mv22 = 0.5 * CHS2 * (nt[3] + nt[4]);
    } else {
        Mv21 = 2.0 / (3.0 * T) * (nt[3] * nt[2] + 2.0 * nt[5] * nt[1]);
        Mv12 = 2.0 / (3.0 * T) * (nt[4] * nt[1] + 2.0 * nt[5] * nt[2]);
        Mv22 = (nt[3] * nt[4] + 2.0 * nt[5] * nt[5]) / T;
    }
    nt[6] = n[6] + om[6] * (Mv21 - n[6]);
    nt[7] = n[7] + om[7] * (Mv12 - n[7]);
    nt[8] = n[8] + om[8] * (Mv22 - n[8]);

    orc_d2q9_step4(nt, ux, uy, rt);
    orc_d2q9_step5(rt, gt);
}

/* ------------------------------------------------------------------------------------------ */
/* Appendix C: D3Q15 energy collision.  Moment order (000, 100, 010, 001, 110, 101, 011, 200,   */
/* 020, 002, 120, 012, 201, 111, 220), Sec. 5.4.                                               */
/* ------------------------------------------------------------------------------------------ */

/* Step 1: raw moments n = P g. */
void orc_d3q15_step1(const double g[15], double r[15])
{
    r[0] = g[0] + g[1] + g[2] + g[3] + g[4] + g[5] + g[6] + g[7] + g[8] + g[9] + g[10] + g[11]
         + g[12] + g[13] + g[14];
    r[1] = g[1] - g[2] + g[7] - g[8] + g[9] - g[10] + g[11] - g[12] + g[13] - g[14];
    r[2] = g[3] - g[4] + g[7] + g[8] - g[9] - g[10] + g[11] + g[12] - g[13] - g[14];
    r[3] = g[5] - g[6] + g[7] + g[8] + g[9] + g[10] - g[11] - g[12] - g[13] - g[14];
    r[4] = g[7] - g[8] - g[9] + g[10] + g[11] - g[12] - g[13] + g[14];
    r[5] = g[7] - g[8] + g[9] - g[10] - g[11] + g[12] - g[13] + g[14];
    r[6] = g[7] + g[8] - g[9] - g[10] - g[11] - g[12] + g[13] + g[14];
    r[7] = g[1] + g[2] + g[7] + g[8] + g[9] + g[10] + g[11] + g[12] + g[13] + g[14];
    r[8] = g[3] + g[4] + g[7] + g[8] + g[9] + g[10] + g[11] + g[12] + g[13] + g[14];
    r[9] = g[5] + g[6] + g[7] + g[8] + g[9] + g[10] + g[11] + g[12] + g[13] + g[14];
    r[10] = g[7] - g[8] + g[9] - g[10] + g[11] - g[12] + g[13] - g[14];
    r[11] = g[7] + g[8] - g[9] - g[10] + g[11] + g[12] - g[13] - g[14];
    r[12] = g[7] + g[8] + g[9] + g[10] - g[11] - g[12] - g[13] - g[14];
    r[13] = g[7] - g[8] - g[9] + g[10] - g[11] + g[12] + g[13] - g[14];
    r[14] = g[7] + g[8] + g[9] + g[10] + g[11] + g[12] + g[13] + g[14];
}

/* Step 2: central moments n^c = F n. */
void orc_d3q15_step2(const double r[15], double ux, double uy, double uz, double c[15])
{
    const double uxx = ux * ux, uyy = uy * uy, uzz = uz * uz;
    c[0] = r[0];
    c[1] = r[1] - ux * r[0];
    c[2] = r[2] - uy * r[0];
    c[3] = r[3] - uz * r[0];
    c[4] = r[4] - ux * r[2] - uy * r[1] + ux * uy * r[0];
    c[5] = r[5] - ux * r[3] - uz * r[1] + ux * uz * r[0];
    c[6] = r[6] - uy * r[3] - uz * r[2] + uy * uz * r[0];
    c[7] = r[7] - 2.0 * ux * r[1] + uxx * r[0];
    c[8] = r[8] - 2.0 * uy * r[2] + uyy * r[0];
    c[9] = r[9] - 2.0 * uz * r[3] + uzz * r[0];
    c[10] = r[10] - ux * r[8] - 2.0 * uy * r[4] + uyy * r[1] + 2.0 * ux * uy * r[2] - ux * uyy * r[0];
    c[11] = r[11] - uy * r[9] - 2.0 * uz * r[6] + uzz * r[2] + 2.0 * uy * uz * r[3] - uy * uzz * r[0];
    c[12] = r[12] - 2.0 * ux * r[5] - uz * r[7] + uxx * r[3] + 2.0 * ux * uz * r[1] - uxx * uz * r[0];
    c[13] = r[13] - ux * r[6] - uy * r[5] - uz * r[4] + ux * uy * r[3] + ux * uz * r[2]
          + uy * uz * r[1] - ux * uy * uz * r[0];
    c[14] = r[14] - 2.0 * ux * r[10] - 2.0 * uy * r[11] + uxx * r[8] + uyy * r[7]
          + 4.0 * ux * uy * r[4] - 2.0 * ux * uyy * r[1] - 2.0 * uxx * uy * r[2] + uxx * uyy * r[0];
}

/* Step 4: raw moments from central moments, n = F^-1 n^c (exact inverse of Step 2). */
void orc_d3q15_step4(const double c[15], double ux, double uy, double uz, double r[15])
{
    const double uxx = ux * ux, uyy = uy * uy, uzz = uz * uz;
    r[0] = c[0];
    r[1] = c[1] + ux * c[0];
    r[2] = c[2] + uy * c[0];
    r[3] = c[3] + uz * c[0];
    r[4] = c[4] + ux * c[2] + uy * c[1] + ux * uy * c[0];
    r[5] = c[5] + ux * c[3] + uz * c[1] + ux * uz * c[0];
    r[6] = c[6] + uy * c[3] + uz * c[2] + uy * uz * c[0];
    r[7] = c[7] + 2.0 * ux * c[1] + uxx * c[0];
    r[8] = c[8] + 2.0 * uy * c[2] + uyy * c[0];
    r[9] = c[9] + 2.0 * uz * c[3] + uzz * c[0];
    r[10] = c[10] + ux * c[8] + 2.0 * uy * c[4] + uyy * c[1] + 2.0 * ux * uy * c[2] + ux * uyy * c[0];
    r[11] = c[11] + uy * c[9] + 2.0 * uz * c[6] + uzz * c[2] + 2.0 * uy * uz * c[3] + uy * uzz * c[0];
    r[12] = c[12] + 2.0 * ux * c[5] + uz * c[7] + uxx * c[3] + 2.0 * ux * uz * c[1] + uxx * uz * c[0];
    r[13] = c[13] + ux * c[6] + uy * c[5] + uz * c[4] + ux * uy * c[3] + ux * uz * c[2]
          + uy * uz * c[1] + ux * uy * uz * c[0];
    r[14] = c[14] + 2.0 * ux * c[10] + 2.0 * uy * c[11] - uyy * c[7] + uxx * c[8] + 2.0 * uyy * c[9]
          + 4.0 * uy * uz * c[6] - 2.0 * ux * uyy * c[1] + 2.0 * uy * uzz * c[2] + 4.0 * uyy * uz * c[3]
          - (uxx * uyy - 2.0 * uyy * uzz) * c[0];
}

/* Step 5: populations from raw moments, g = P^-1 n. */
void orc_d3q15_step5(const double r[15], double g[15])
{
    g[0] = r[0] - r[9] - r[8] - r[7] + 2.0 * r[14];
    g[1] = (r[1] - r[10] + r[7] - r[14]) / 2.0;
    g[2] = (r[10] - r[1] + r[7] - r[14]) / 2.0;
    g[3] = (r[2] - r[11] + r[8] - r[14]) / 2.0;
    g[4] = (r[11] - r[2] + r[8] - r[14]) / 2.0;
    g[5] = (r[3] + r[9] - r[12] - r[14]) / 2.0;
    g[6] = (r[9] - r[3] + r[12] - r[14]) / 2.0;
    g[7] = (r[6] + r[11] + r[5] + r[4] + r[13] + r[10] + r[12] + r[14]) / 8.0;
    g[8] = (r[6] + r[11] - r[5] - r[4] - r[13] - r[10] + r[12] + r[14]) / 8.0;
    g[9] = (r[5] - r[11] - r[6] - r[4] - r[13] + r[10] + r[12] + r[14]) / 8.0;
    g[10] = (r[4] - r[11] - r[5] - r[6] + r[13] - r[10] + r[12] + r[14]) / 8.0;
    g[11] = (r[11] - r[6] - r[5] + r[4] - r[13] + r[10] - r[12] + r[14]) / 8.0;
    g[12] = (r[11] - r[6] + r[5] - r[4] + r[13] - r[10] - r[12] + r[14]) / 8.0;
    g[13] = (r[6] - r[11] - r[5] - r[4] + r[13] + r[10] - r[12] + r[14]) / 8.0;
    g[14] = (r[6] - r[11] + r[5] + r[4] - r[13] - r[10] - r[12] + r[14]) / 8.0;
}

/*
 * Appendix C, Steps 1-5: D3Q15 energy collision.  om[0..14] are the paper's omega_0..omega_14.
 * option 0 takes the option-A attractors of orders 3-4 (Eq. g-attractorsD3Q15optionA, reading
 * R3), option 1 the renormalized option-B list that follows it in Sec. 5.3, both from the
 * post-collision moments of orders 0-2.
 */
void orc_d3q15_g_collide(const double g[15], double ux, double uy, double uz, const double om[15],
                         int option, double gt[15])
{
    double r[15], n[15], nt[15], rt[15];
    orc_d3q15_step1(g, r);
    orc_d3q15_step2(r, ux, uy, uz, n);

    const double T = n[0];
    double Mv[15];
    Mv[0] = T;
    Mv[1] = 0.0;
    Mv[2] = 0.0;
    Mv[3] = 0.0;
    Mv[4] = 0.0;
    Mv[5] = 0.0;
    Mv[6] = 0.0;
    Mv[7] = CHS2 * T;
    Mv[8] = CHS2 * T;
    Mv[9] = CHS2 * T;
    for (int j = 0; j <= 9; ++j) nt[j] = n[j] + om[j] * (Mv[j] - n[j]);

    if (option == 0) {
        Mv[10] = (2.0 / 3.0) * CHS2 * nt[1];
        Mv[11] = (2.0 / 3.0) * CHS2 * nt[2];
        Mv[12] = (2.0 / 3.0) * CHS2 * nt[3];
        Mv[13] = 0.0;
        Mv[14] = 0.5 * CHS2 * (nt[7] + nt[8]);
    } else {
        /* moment slots: 1 = 100, 2 = 010, 3 = 001, 4 = 110, 5 = 101, 6 = 011, 7 = 200,
         * 8 = 020, 9 = 002 */
        const double c = 2.0 / (3.0 * T);
        Mv[10] = c * (nt[8] * nt[1] + 2.0 * nt[4] * nt[2]);                  /* 120 */
        Mv[11] = c * (nt[9] * nt[2] + 2.0 * nt[6] * nt[3]);                  /* 012 */
        Mv[12] = c * (nt[7] * nt[3] + 2.0 * nt[5] * nt[1]);                  /* 201 */
        Mv[13] = c * (nt[4] * nt[3] + nt[6] * nt[1] + nt[5] * nt[2]);        /* 111 */
        Mv[14] = (nt[7] * nt[8] + 2.0 * nt[4] * nt[4]) / T;                  /* 220 */
    }
    for (int j = 10; j <= 14; ++j) nt[j] = n[j] + om[j] * (Mv[j] - n[j]);

    orc_d3q15_step4(nt, ux, uy, uz, rt);
    orc_d3q15_step5(rt, gt);
}

/* ------------------------------------------------------------------------------------------ */
/* D3Q27 flow collision (Sec. 5.1-5.2, reading R6).                                            */
/* ------------------------------------------------------------------------------------------ */

/* Central moments by their definition: kappa_mnp = sum_a f_a (e_ax-ux)^m (e_ay-uy)^n (e_az-uz)^p. */
void orc_d3q27_central(const double f[27], double ux, double uy, double uz, double k[27])
{
    for (int j = 0; j < 27; ++j) {
        double s = 0.0;
        for (int a = 0; a < 27; ++a)
            s += f[a] * ipow(D3Q27_E[a][0] - ux, M27[j][0]) * ipow(D3Q27_E[a][1] - uy, M27[j][1])
               * ipow(D3Q27_E[a][2] - uz, M27[j][2]);
        k[j] = s;
    }
}

/* Raw moments from central moments by the binomial expansion of e^m = ((e - u) + u)^m. */
void orc_d3q27_raw_from_central(const double k[27], double ux, double uy, double uz, double r[27])
{
    for (int j = 0; j < 27; ++j) {
        const int m = M27[j][0], n = M27[j][1], p = M27[j][2];
        double s = 0.0;
        for (int i = 0; i <= m; ++i)
            for (int l = 0; l <= n; ++l)
                for (int q = 0; q <= p; ++q)
                    s += binom(m, i) * binom(n, l) * binom(p, q) * ipow(ux, m - i)
                       * ipow(uy, n - l) * ipow(uz, p - q) * k[k27_index(i, l, q)];
        r[j] = s;
    }
}

/* P for D3Q27: P[j][a] = e_ax^m e_ay^n e_az^p over the 27 monomials of Sec. 5.2. */
static double P27[27][27], P27INV[27][27];
static int P27_ready = 0;

static void d3q27_build_inverse(void)
{
    /* Gauss-Jordan elimination with partial pivoting on [P | I]. */
    double a[27][54];
    for (int j = 0; j < 27; ++j)
        for (int c = 0; c < 27; ++c) {
            P27[j][c] = ipow(D3Q27_E[c][0], M27[j][0]) * ipow(D3Q27_E[c][1], M27[j][1])
                      * ipow(D3Q27_E[c][2], M27[j][2]);
            a[j][c] = P27[j][c];
            a[j][27 + c] = (j == c) ? 1.0 : 0.0;
        }
    for (int col = 0; col < 27; ++col) {
        int piv = col;
        for (int r = col + 1; r < 27; ++r)
            if (fabs(a[r][col]) > fabs(a[piv][col])) piv = r;
        if (piv != col)
            for (int c = 0; c < 54; ++c) {
                double t = a[col][c];
                a[col][c] = a[piv][c];
                a[piv][c] = t;
            }
        const double d = a[col][col];
        for (int c = 0; c < 54; ++c) a[col][c] /= d;
        for (int r = 0; r < 27; ++r) {
            if (r == col || a[r][col] == 0.0) continue;
            const double m = a[r][col];
            for (int c = 0; c < 54; ++c) a[r][c] -= m * a[col][c];
        }
    }
    for (int j = 0; j < 27; ++j)
        for (int c = 0; c < 27; ++c) P27INV[j][c] = a[j][27 + c];
    P27_ready = 1;
}

/* Must be called once before any D3Q27 call (not thread-safe itself; orc_create calls it). */
void orc_d3q27_init(void)
{
    if (!P27_ready) d3q27_build_inverse();
}

void orc_d3q27_raw(const double f[27], double r[27])
{
    orc_d3q27_init();
    for (int j = 0; j < 27; ++j) {
        double s = 0.0;
        for (int a = 0; a < 27; ++a) s += P27[j][a] * f[a];
        r[j] = s;
    }
}

void orc_d3q27_pop_from_raw(const double r[27], double f[27])
{
    orc_d3q27_init();
    for (int a = 0; a < 27; ++a) {
        double s = 0.0;
        for (int j = 0; j < 27; ++j) s += P27INV[a][j] * r[j];
        f[a] = s;
    }
}

void orc_d3q27_macro(const double f[27], double Fx, double Fy, double Fz, double out[4])
{
    double rho = 0.0, jx = 0.0, jy = 0.0, jz = 0.0;
    for (int a = 0; a < 27; ++a) {
        rho += f[a];
        jx += f[a] * D3Q27_E[a][0];
        jy += f[a] * D3Q27_E[a][1];
        jz += f[a] * D3Q27_E[a][2];
    }
    out[0] = rho;
    out[1] = (jx + 0.5 * Fx) / rho;
    out[2] = (jy + 0.5 * Fy) / rho;
    out[3] = (jz + 0.5 * Fz) / rho;
}

/* Attractors of orders 4-6 (Sec. 5.2 discrete list, reading R4) from post-collision kt[]. */
void orc_d3q27_attractors_high(const double kt[27], double rho, double Mv[27])
{
    for (int j = 0; j < 27; ++j) Mv[j] = 0.0;
    Mv[K220] = (kt[K200] * kt[K020] + 2.0 * kt[K110] * kt[K110]) / rho;
    Mv[K202] = (kt[K200] * kt[K002] + 2.0 * kt[K101] * kt[K101]) / rho;
    Mv[K022] = (kt[K020] * kt[K002] + 2.0 * kt[K011] * kt[K011]) / rho;
    Mv[K211] = (kt[K200] * kt[K011] + 2.0 * kt[K110] * kt[K101]) / rho;
    Mv[K121] = (kt[K020] * kt[K101] + 2.0 * kt[K110] * kt[K011]) / rho;
    Mv[K112] = (kt[K002] * kt[K110] + 2.0 * kt[K011] * kt[K101]) / rho;
    Mv[K122] = 2.0 / (5.0 * rho)
             * (kt[K020] * kt[K102] + kt[K002] * kt[K120] + 4.0 * kt[K011] * kt[K111]
                + 2.0 * (kt[K101] * kt[K021] + kt[K110] * kt[K012]));
    Mv[K212] = 2.0 / (5.0 * rho)
             * (kt[K200] * kt[K012] + kt[K002] * kt[K210] + 4.0 * kt[K101] * kt[K111]
                + 2.0 * (kt[K110] * kt[K102] + kt[K011] * kt[K201]));
    Mv[K221] = 2.0 / (5.0 * rho)
             * (kt[K200] * kt[K021] + kt[K020] * kt[K201] + 4.0 * kt[K110] * kt[K111]
                + 2.0 * (kt[K011] * kt[K210] + kt[K101] * kt[K120]));
    Mv[K222] = 1.0 / (3.0 * rho)
             * (kt[K200] * kt[K022] + kt[K020] * kt[K202] + kt[K002] * kt[K220]
                + 4.0 * (kt[K110] * kt[K112] + kt[K101] * kt[K121] + kt[K011] * kt[K211]));
}

/*
 * D3Q27 flow collision, reading R6.  om[j] is the rate of the j-th entry of m^c in the order
 * of Sec. 5.2, except for the three diagonal second-order slots: om[K200] relaxes the trace
 * kappa_200 + kappa_020 + kappa_002 (bulk), om[K020] the deviator kappa_200 - kappa_020 and
 * om[K002] the deviator kappa_200 - kappa_002 (shear).  Sources follow Eq. forcing:3D with the
 * pre-collision central moments; second-order sources are zero (reading R5); delta_t = 1.
 */
void orc_d3q27_f_collide(const double f[27], double rho, double ux, double uy, double uz,
                         double Fx, double Fy, double Fz, const double om[27], double ft[27])
{
    double k[27], kt[27], Mv[27], sg[27], rt[27];
    orc_d3q27_central(f, ux, uy, uz, k);

    /* Sources sigma_mnp. */
    for (int j = 0; j < 27; ++j) {
        const int m = M27[j][0], n = M27[j][1], p = M27[j][2];
        const int order = m + n + p;
        double s = 0.0;
        if (order == 1) {
            s = m * Fx + n * Fy + p * Fz; /* kappa_000 = rho */
        } else if (order >= 3) {
            if (m > 0) s += m * (Fx / rho) * k[k27_index(m - 1, n, p)];
            if (n > 0) s += n * (Fy / rho) * k[k27_index(m, n - 1, p)];
            if (p > 0) s += p * (Fz / rho) * k[k27_index(m, n, p - 1)];
        }
        sg[j] = s;
    }

    /* Orders 0-1 (attractors rho, 0, 0, 0). */
    kt[K000] = k[K000] + om[K000] * (rho - k[K000]) + (1.0 - om[K000] / 2.0) * sg[K000];
    for (int j = K100; j <= K001; ++j)
        kt[j] = k[j] + om[j] * (0.0 - k[j]) + (1.0 - om[j] / 2.0) * sg[j];

    /* Order 2: off-diagonal toward 0, trace toward 3 c_s^2 rho, deviators toward 0. */
    for (int j = K110; j <= K011; ++j)
        kt[j] = k[j] + om[j] * (0.0 - k[j]) + (1.0 - om[j] / 2.0) * sg[j];
    const double tr = k[K200] + k[K020] + k[K002];
    const double d1 = k[K200] - k[K020];
    const double d2 = k[K200] - k[K002];
    const double trt = tr + om[K200] * (3.0 * CS2 * rho - tr);
    const double d1t = d1 + om[K020] * (0.0 - d1);
    const double d2t = d2 + om[K002] * (0.0 - d2);
    kt[K200] = (trt + d1t + d2t) / 3.0;
    kt[K020] = (trt - 2.0 * d1t + d2t) / 3.0;
    kt[K002] = (trt + d1t - 2.0 * d2t) / 3.0;

    /* Order 3: attractors are zero. */
    for (int j = K120; j <= K111; ++j)
        kt[j] = k[j] + om[j] * (0.0 - k[j]) + (1.0 - om[j] / 2.0) * sg[j];

    /* Order 4 (from post-collision order 2), then 5 (orders 2-3), then 6 (orders 2 and 4). */
    orc_d3q27_attractors_high(kt, rho, Mv);
    for (int j = K220; j <= K112; ++j)
        kt[j] = k[j] + om[j] * (Mv[j] - k[j]) + (1.0 - om[j] / 2.0) * sg[j];
    orc_d3q27_attractors_high(kt, rho, Mv);
    for (int j = K122; j <= K221; ++j)
        kt[j] = k[j] + om[j] * (Mv[j] - k[j]) + (1.0 - om[j] / 2.0) * sg[j];
    orc_d3q27_attractors_high(kt, rho, Mv);
    kt[K222] = k[K222] + om[K222] * (Mv[K222] - k[K222]) + (1.0 - om[K222] / 2.0) * sg[K222];

    orc_d3q27_raw_from_central(kt, ux, uy, uz, rt);
    orc_d3q27_pop_from_raw(rt, ft);
}

/* ------------------------------------------------------------------------------------------ */
/* Rest-state attractor populations (used for initial states and the anti-bounce-back weight). */
/* ------------------------------------------------------------------------------------------ */

/* Flow populations whose central moments are the attractor at density rho and velocity u. */
void orc_equilibrium_f(int dim, double rho, double ux, double uy, double uz, double *out)
{
    if (dim == 2) {
        double c[9] = {rho, 0, 0, CS2 * rho, CS2 * rho, 0, 0, 0, 0}, r[9];
        c[8] = (c[3] * c[4] + 2.0 * c[5] * c[5]) / rho;
        orc_d2q9_step4(c, ux, uy, r);
        orc_d2q9_step5(r, out);
    } else {
        double c[27] = {0}, Mv[27], r[27];
        c[K000] = rho;
        c[K200] = c[K020] = c[K002] = CS2 * rho;
        orc_d3q27_attractors_high(c, rho, Mv);
        for (int j = K220; j <= K112; ++j) c[j] = Mv[j];
        orc_d3q27_attractors_high(c, rho, Mv);
        for (int j = K122; j <= K221; ++j) c[j] = Mv[j];
        orc_d3q27_attractors_high(c, rho, Mv);
        c[K222] = Mv[K222];
        orc_d3q27_raw_from_central(c, ux, uy, uz, r);
        orc_d3q27_pop_from_raw(r, out);
    }
}

/* Energy populations whose central moments are the option-A attractor at T and velocity u. */
void orc_equilibrium_g(int dim, double T, double ux, double uy, double uz, double *out)
{
    if (dim == 2) {
        double c[9] = {T, 0, 0, CHS2 * T, CHS2 * T, 0, 0, 0, 0}, r[9];
        c[6] = (2.0 / 3.0) * CHS2 * c[2];
        c[7] = (2.0 / 3.0) * CHS2 * c[1];
        c[8] = 0.5 * CHS2 * (c[3] + c[4]);
        orc_d2q9_step4(c, ux, uy, r);
        orc_d2q9_step5(r, out);
    } else {
        double c[15] = {T, 0, 0, 0, 0, 0, 0, CHS2 * T, CHS2 * T, CHS2 * T, 0, 0, 0, 0, 0}, r[15];
        c[10] = (2.0 / 3.0) * CHS2 * c[1];
        c[11] = (2.0 / 3.0) * CHS2 * c[2];
        c[12] = (2.0 / 3.0) * CHS2 * c[3];
        c[14] = 0.5 * CHS2 * (c[7] + c[8]);
        orc_d3q15_step4(c, ux, uy, uz, r);
        orc_d3q15_step5(r, out);
    }
}

/* ------------------------------------------------------------------------------------------ */
/* Grid: collide-and-stream on a box with periodic axes and half-way walls.                    */
/* The stored state is the post-collision populations f~, g~ (before streaming).              */
/* ------------------------------------------------------------------------------------------ */

typedef struct {
    int dim, nx, ny, nz, qf, qg;
    long n;
    int face_bc[6];
    double T_wall[6];
    double *profile[6];
    double gbeta, T_ref;
    int gravity_axis;
    double om_f[27], om_g[15];
    int g_option;              /* energy attractors of orders 3-4: 0 = option A, 1 = option B */
    double wg[15];
    const int (*ef)[3];
    const int (*eg)[3];
    int opp_f[27], opp_g[15];
    double *f, *g, *f2, *g2;
} orc_grid;

static int find_opp(const int (*e)[3], int q, int a)
{
    for (int b = 0; b < q; ++b)
        if (e[b][0] == -e[a][0] && e[b][1] == -e[a][1] && e[b][2] == -e[a][2]) return b;
    return -1;
}

orc_grid *orc_create(int dim, int nx, int ny, int nz)
{
    if (dim != 2 && dim != 3) return NULL;
    if (dim == 2) nz = 1;
    orc_d3q27_init();
    orc_grid *G = (orc_grid *)calloc(1, sizeof(orc_grid));
    G->dim = dim;
    G->nx = nx;
    G->ny = ny;
    G->nz = nz;
    G->n = (long)nx * ny * nz;
    G->qf = dim == 2 ? 9 : 27;
    G->qg = dim == 2 ? 9 : 15;
    G->ef = dim == 2 ? D2Q9_E : D3Q27_E;
    G->eg = dim == 2 ? D2Q9_E : D3Q15_E;
    for (int a = 0; a < G->qf; ++a) G->opp_f[a] = find_opp(G->ef, G->qf, a);
    for (int a = 0; a < G->qg; ++a) G->opp_g[a] = find_opp(G->eg, G->qg, a);
    for (int a = 0; a < 27; ++a) G->om_f[a] = 1.0;
    for (int a = 0; a < 15; ++a) G->om_g[a] = 1.0;
    orc_equilibrium_g(dim, 1.0, 0.0, 0.0, 0.0, G->wg);
    for (int i = 0; i < 6; ++i) G->face_bc[i] = ORC_PERIODIC;
    G->gravity_axis = dim == 2 ? 1 : 2;
    G->f = (double *)calloc((size_t)G->qf * G->n, sizeof(double));
    G->g = (double *)calloc((size_t)G->qg * G->n, sizeof(double));
    G->f2 = (double *)calloc((size_t)G->qf * G->n, sizeof(double));
    G->g2 = (double *)calloc((size_t)G->qg * G->n, sizeof(double));
    return G;
}

void orc_destroy(orc_grid *G)
{
    if (!G) return;
    for (int i = 0; i < 6; ++i) free(G->profile[i]);
    free(G->f);
    free(G->g);
    free(G->f2);
    free(G->g2);
    free(G);
}

void orc_set_bc(orc_grid *G, const int face_bc[6], const double T_wall[6], double T_ref,
                int gravity_axis, double gbeta)
{
    for (int i = 0; i < 6; ++i) {
        G->face_bc[i] = face_bc[i];
        G->T_wall[i] = T_wall[i];
    }
    G->T_ref = T_ref;
    G->gravity_axis = gravity_axis;
    G->gbeta = gbeta;
}

void orc_set_g_option(orc_grid *G, int option) { G->g_option = option ? 1 : 0; }

void orc_set_omegas(orc_grid *G, const double *om_f, const double *om_g)
{
    for (int a = 0; a < G->qf; ++a) G->om_f[a] = om_f[a];
    for (int a = 0; a < G->qg; ++a) G->om_g[a] = om_g[a];
}

/* Number of nodes on a face (its tangential extent). */
static long face_nodes(const orc_grid *G, int face)
{
    const int ax = face / 2;
    if (ax == 0) return (long)G->ny * G->nz;
    if (ax == 1) return (long)G->nx * G->nz;
    return (long)G->nx * G->ny;
}

/* Tangential index of node (x, y, z) on a face of the given axis. */
static long face_index(const orc_grid *G, int face, int x, int y, int z)
{
    const int ax = face / 2;
    if (ax == 0) return y + (long)G->ny * z;
    if (ax == 1) return x + (long)G->nx * z;
    return x + (long)G->nx * y;
}

int orc_set_wall_profile(orc_grid *G, int face, const double *Tw, long n)
{
    if (face < 0 || face > 5 || n != face_nodes(G, face)) return -1;
    free(G->profile[face]);
    G->profile[face] = (double *)malloc(sizeof(double) * n);
    memcpy(G->profile[face], Tw, sizeof(double) * n);
    return 0;
}

static double wall_T(const orc_grid *G, int face, int x, int y, int z)
{
    if (G->profile[face]) return G->profile[face][face_index(G, face, x, y, z)];
    return G->T_wall[face];
}

void orc_set_state(orc_grid *G, const double *f, const double *g)
{
    memcpy(G->f, f, sizeof(double) * G->qf * G->n);
    memcpy(G->g, g, sizeof(double) * G->qg * G->n);
}

void orc_get_state(const orc_grid *G, double *f, double *g)
{
    memcpy(f, G->f, sizeof(double) * G->qf * G->n);
    memcpy(g, G->g, sizeof(double) * G->qg * G->n);
}

/*
 * Source node of the link arriving at (x, y, z) along e, after wrapping periodic axes.
 * Returns -1 if the source lies beyond a wall.  A link across an edge or corner of the box
 * crosses two or three walls; the one that decides its rule is the crossed face that comes last
 * in the order -z, -y, -x, +x, +y, +z (reading R7).  *fixed is that face when it has a fixed
 * temperature (anti-bounce-back), else -1 (bounce-back).
 */
static int face_rank(int face)
{
    static const int rank[6] = {2, 3, 1, 4, 0, 5};   /* -x, +x, -y, +y, -z, +z */
    return rank[face];
}

static long link_source(const orc_grid *G, int x, int y, int z, const int e[3], int *fixed)
{
    int s[3] = {x - e[0], y - e[1], z - e[2]};
    const int ext[3] = {G->nx, G->ny, G->nz};
    int decide = -1;
    *fixed = -1;
    for (int ax = 0; ax < G->dim; ++ax) {
        int face = -1;
        if (s[ax] < 0) face = 2 * ax;
        if (s[ax] >= ext[ax]) face = 2 * ax + 1;
        if (face < 0) continue;
        if (G->face_bc[face] == ORC_PERIODIC) {
            s[ax] = (s[ax] + ext[ax]) % ext[ax];
            continue;
        }
        if (decide < 0 || face_rank(face) > face_rank(decide)) decide = face;
    }
    if (decide >= 0) {
        if (G->face_bc[decide] == ORC_WALL_FIXED_T) *fixed = decide;
        return -1;
    }
    return s[0] + (long)G->nx * (s[1] + (long)G->ny * s[2]);
}

/* Streaming step (Eqs. LBMsteps-stream, LBMsteps-streamg) with the Sec. 6.1 wall rules. */
static void pull_node(const orc_grid *G, int x, int y, int z, double *fo, double *go)
{
    const long i = x + (long)G->nx * (y + (long)G->ny * z);
    for (int a = 0; a < G->qf; ++a) {
        int fixed;
        const long s = link_source(G, x, y, z, G->ef[a], &fixed);
        fo[a] = s >= 0 ? G->f[(long)a * G->n + s] : G->f[(long)G->opp_f[a] * G->n + i];
    }
    for (int a = 0; a < G->qg; ++a) {
        int fixed;
        const long s = link_source(G, x, y, z, G->eg[a], &fixed);
        if (s >= 0) {
            go[a] = G->g[(long)a * G->n + s];
        } else {
            const double back = G->g[(long)G->opp_g[a] * G->n + i];
            go[a] = fixed >= 0 ? -back + 2.0 * G->wg[a] * wall_T(G, fixed, x, y, z) : back;
        }
    }
}

static void node_update(orc_grid *G, int x, int y, int z)
{
    const long i = x + (long)G->nx * (y + (long)G->ny * z);
    double fo[27], go[15], ft[27], gt[15];
    pull_node(G, x, y, z, fo, go);

    double T = 0.0;
    for (int a = 0; a < G->qg; ++a) T += go[a];
    double F[3] = {0.0, 0.0, 0.0};
    F[G->gravity_axis] = G->gbeta * (T - G->T_ref);

    if (G->dim == 2) {
        double mac[3];
        orc_d2q9_macro(fo, F[0], F[1], mac);
        orc_d2q9_f_collide(fo, mac[0], mac[1], mac[2], F[0], F[1], G->om_f, ft);
        orc_d2q9_g_collide(go, mac[1], mac[2], G->om_g, G->g_option, gt);
    } else {
        double mac[4];
        orc_d3q27_macro(fo, F[0], F[1], F[2], mac);
        orc_d3q27_f_collide(fo, mac[0], mac[1], mac[2], mac[3], F[0], F[1], F[2], G->om_f, ft);
        orc_d3q15_g_collide(go, mac[1], mac[2], mac[3], G->om_g, G->g_option, gt);
    }
    for (int a = 0; a < G->qf; ++a) G->f2[(long)a * G->n + i] = ft[a];
    for (int a = 0; a < G->qg; ++a) G->g2[(long)a * G->n + i] = gt[a];
}

void orc_step(orc_grid *G, long nsteps)
{
    for (long t = 0; t < nsteps; ++t) {
#pragma omp parallel for collapse(2) schedule(static)
        for (int z = 0; z < G->nz; ++z)
            for (int y = 0; y < G->ny; ++y)
                for (int x = 0; x < G->nx; ++x) node_update(G, x, y, z);
        double *t1 = G->f;
        G->f = G->f2;
        G->f2 = t1;
        double *t2 = G->g;
        G->g = G->g2;
        G->g2 = t2;
    }
}

/* Step a restricted box [x0,x1) x [y0,y1) x [z0,z1) once, without swapping (timing samples). */
void orc_update_box(orc_grid *G, int x0, int x1, int y0, int y1, int z0, int z1)
{
#pragma omp parallel for collapse(2) schedule(static)
    for (int z = z0; z < z1; ++z)
        for (int y = y0; y < y1; ++y)
            for (int x = x0; x < x1; ++x) node_update(G, x, y, z);
}

int orc_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Fields rho, u, T of the streamed populations f(x, t), g(x, t) (Step 7 of App. A/B/C). */
void orc_fields(const orc_grid *G, double *rho, double *ux, double *uy, double *uz, double *T)
{
    for (int z = 0; z < G->nz; ++z)
        for (int y = 0; y < G->ny; ++y)
            for (int x = 0; x < G->nx; ++x) {
                const long i = x + (long)G->nx * (y + (long)G->ny * z);
                double fo[27], go[15];
                pull_node(G, x, y, z, fo, go);
                double t = 0.0;
                for (int a = 0; a < G->qg; ++a) t += go[a];
                double F[3] = {0.0, 0.0, 0.0};
                F[G->gravity_axis] = G->gbeta * (t - G->T_ref);
                double r = 0.0, j[3] = {0.0, 0.0, 0.0};
                for (int a = 0; a < G->qf; ++a) {
                    r += fo[a];
                    for (int d = 0; d < 3; ++d) j[d] += fo[a] * G->ef[a][d];
                }
                rho[i] = r;
                ux[i] = (j[0] + 0.5 * F[0]) / r;
                uy[i] = (j[1] + 0.5 * F[1]) / r;
                uz[i] = (j[2] + 0.5 * F[2]) / r;
                T[i] = t;
            }
}

/*
 * Local wall Nusselt numbers on a fixed-temperature face (Sec. 6.1): the wall-normal derivative
 * at the wall from the second-order Lagrange polynomial through the wall (x0 = 0) and the first two
 * node layers (x1 = 1/2, x2 = 3/2), dT/dn = -8/3 T_w + 3 T_1 - 1/3 T_2, with n pointing into the
 * fluid.  Nu = -sgn (L / dT) dT/dn, sgn = +1 on a face at or above T_ref (heat enters the fluid)
 * and -1 below it, so that Nu > 0 on both the hot and the cold wall.
 * Writes face_nodes values (tangential order of face_index) and returns 0, or -1 on a bad face.
 */
int orc_nusselt(const orc_grid *G, int face, double L, double dT, double *nu)
{
    if (face < 0 || face / 2 >= G->dim || G->face_bc[face] != ORC_WALL_FIXED_T) return -1;
    const int ax = face / 2, hi = face & 1;
    const int ext[3] = {G->nx, G->ny, G->nz};
    if (ext[ax] < 2) return -1;
    const double sgn = G->T_wall[face] >= G->T_ref ? 1.0 : -1.0;
    for (int z = 0; z < G->nz; ++z)
        for (int y = 0; y < G->ny; ++y)
            for (int x = 0; x < G->nx; ++x) {
                int c[3] = {x, y, z};
                if (c[ax] != (hi ? ext[ax] - 1 : 0)) continue;
                double Tl[2];
                for (int l = 0; l < 2; ++l) {
                    int p[3] = {x, y, z};
                    p[ax] = hi ? ext[ax] - 1 - l : l;
                    double fo[27], go[15], t = 0.0;
                    pull_node(G, p[0], p[1], p[2], fo, go);
                    for (int a = 0; a < G->qg; ++a) t += go[a];
                    Tl[l] = t;
                }
                const double Tw = wall_T(G, face, x, y, z);
                const double dTdn = -8.0 / 3.0 * Tw + 3.0 * Tl[0] - 1.0 / 3.0 * Tl[1];
                nu[face_index(G, face, x, y, z)] = -sgn * (L / dT) * dTdn;
            }
    return 0;
}

/* splitmix64 (Steele, Lea & Flood 2014): the i-th output of the stream seeded with `seed`. */
uint64_t orc_splitmix64(uint64_t seed, uint64_t i)
{
    uint64_t z = seed + (i + 1) * 0x9e3779b97f4a7c15ULL;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

/* Uniform double in [0, 1) from the top 53 bits of the i-th splitmix64 output. */
double orc_uniform01(uint64_t seed, uint64_t i)
{
    return (double)(orc_splitmix64(seed, i) >> 11) * (1.0 / 9007199254740992.0);
}

/*
 * Initial state: fluid at rest at density 1 and temperature T_init + perturb * (2 U_i - 1),
 * U_i the i-th uniform of the splitmix64 stream, i the linear node index (x fastest).
 * Populations are the rest-state attractors; they are stored as the post-collision state.
 */
void orc_init_rest(orc_grid *G, double T_init, uint64_t seed, double perturb)
{
    double fe[27], ge[15];
    orc_equilibrium_f(G->dim, 1.0, 0.0, 0.0, 0.0, fe);
    for (long i = 0; i < G->n; ++i) {
        const double T = T_init + (perturb != 0.0 ? perturb * (2.0 * orc_uniform01(seed, i) - 1.0) : 0.0);
        orc_equilibrium_g(G->dim, T, 0.0, 0.0, 0.0, ge);
        for (int a = 0; a < G->qf; ++a) G->f[(long)a * G->n + i] = fe[a];
        for (int a = 0; a < G->qg; ++a) G->g[(long)a * G->n + i] = ge[a];
    }
}
