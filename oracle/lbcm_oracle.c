/*
 * lbcm_oracle.c -- plain FP64 CPU oracle for one time step of the colour-gradient
 * lattice Boltzmann model with nonorthogonal central moments (Saito, De Rosis,
 * Festuccia, Kaneko, Abe, Koyama, arXiv:1804.08923, Section II).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, literal reference that the
 * CUDA path is checked against.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark load it; the product library never does.  It
 * shares no code, header, table or helper with the CUDA path.
 *
 * Every step follows the paper's equations in the paper's order with dense
 * 27x27 matrices:
 *   - velocity set c_i                       Eq. (8)
 *   - LB equation, operator split            Eq. (9) and the Omega^(3)[Omega^(1)+Omega^(2)] split
 *   - GMRT collision -T^-1 K T (f - f^e) + F Eq. (11) with T = N M (Eq. (14))
 *   - densities, Guo momentum                Eq. (13)
 *   - relaxation matrix K, nu(s_2nu)         Eq. (16), text below Eq. (17)
 *   - enhanced equilibrium, varphi_i, Phi_i  Eqs. (18), (20), (21), G tensor Eq. (24)
 *   - order parameter, alpha-bar, nu-bar     Eq. (23), harmonic mean Eq. (22), alpha-bar Eq. (27)
 *   - forcing                                Eqs. (28), (29)
 *   - perturbation, B_i, sigma               Eqs. (30), (31), (32)
 *   - recolouring                            Eqs. (33), (34)
 *   - isotropic gradient                     Eq. (40), the 27-point central scheme of Section II
 *   - inlet / free-slip / convective outflow Section IV.A (Lou-type implicit convective scheme)
 *   - body force F = (rho - rho_b^0) g       Eq. (48)
 *   - static droplet initial state           Section III
 *
 * Readings of passages the paper leaves open (the same on the CUDA side):
 *   R1  Eq. (30) prints the numerator (c_i . grad phi) unsquared; the squared
 *       form is used (the only form with zero mass and momentum).
 *   R2  The perturbation is applied for each colour k = r, b with A_r = A_b = A, so the
 *       colour-blind population receives the sum of both; with the capillary stress
 *       S = -tau sum_i sum_k Omega_i^k(2) c_i c_i this is the form for which
 *       sigma = (4/9) A tau (Eq. (32)) holds.
 *   R3  |grad phi| in Eqs. (30) and cos(theta_i) is regularised as
 *       sqrt(|grad phi|^2 + eps^2); cos(theta_0) = 0.
 *   R4  A = 9 sigma / (4 tau) per node with tau = 1/s_2nu(x).
 *   R5  grad rho in Phi_i and G uses the total density rho.
 *   R6  f^(e)(rho, 0) in the recolouring is rho varphi_i(alpha-bar) (Phi vanishes at u = 0).
 *   R7  Inlet (z = 0, ghost plane z = -1): unknown populations (c_iz = +1) of node
 *       (x, y, 0) come from the ghost at (x - c_ix, y - c_iy, -1).  Inside the disc
 *       (x - x_c)^2 + (y - y_c)^2 < (D/2)^2, with x_c = (nx - 1)/2, that is the red
 *       equilibrium f^(e)(rho_r^0, u_in) with alpha_r and Phi = 0, and zero blue;
 *       elsewhere the half-way specular (free-slip) mirror S_{m(i)}(x - c_ix, y - c_iy, 0)
 *       where m flips c_z.  u_in = u_j0 (a xi rhat_x, a xi rhat_y, 1), xi in [-1, 1)
 *       from SplitMix64 of (seed, step, x, y); a = 0 gives the paper's undisturbed inlet.
 *   R8  Convective outflow at z = N = nz - 1 (Eqs. (45)-(47)) acts on all 27 post-stream
 *       populations of both colours; lambda = U_c(t + 1) = u_z(x, y, N - 1, t + 1) as Eqs. (46)
 *       and (47) give it, clamped to [0, 1] (the paper is silent on backflow).
 *   R9  Gradient ghosts: z = -1 is phi = 1, rho = rho_r^0 inside the inlet disc and the
 *       mirror of z = 0 elsewhere (or on a free-slip wall); z = N + 1 mirrors z = N.
 *   R10 Initial populations from fields (rho_r, rho_b, u):
 *       f_i^k = rho_k [varphi_i(alpha_k) + w_i(3 cu + 9/2 cu^2 - 3/2 u^2 + 9/2 cu^3 - 9/2 cu u^2)].
 *   R11 Inlet profile (not in the paper, whose inlet is uniform; the parameters the
 *       adjoint differentiates): u_z = u_j0 [1 + sum_{m=1..8} (a_m cos m theta + b_m sin m theta)]
 *       with theta the polar angle of the source column about the disc centre (0 at the centre).
 *   R14 Free-slip side walls (Section IV.A: walls cover the sides, free slip): at x = -1/2 and
 *       x = nx - 1/2 (likewise y) a pull whose source lies beyond the wall reads the node's own
 *       layer with that velocity component reversed (half-way specular reflection); the z rules
 *       then act on the reflected direction at the reflected source column.  Gradient ghosts
 *       beyond a side wall mirror the wall layer; fragments and the area objective do not wrap
 *       across it.
 *   R15 Alternative to the printed alpha-bar interpolation (alpha_mix = 1): weights rho_k / rho
 *       (mass fractions) instead of (1 +- phi)/2 (volume fractions), which makes the equation
 *       of state additive, rho c_s^2(alpha-bar) = rho_r c_r^2 + rho_b c_b^2.  Not the paper's
 *       formula; the reading under which its density-ratio droplets stay stable.
 *   R13 Fragments (Section IV.B, diameter procedure): the jet region is phi > 0 of the state's
 *       colour densities; fragments are its connected components with face (6) or full (26)
 *       neighbourhoods, wrapping where the lattice is periodic; V = node count, d = (6V/pi)^(1/3);
 *       the continuous column from the nozzle is every component with a node on z = 0 (inlet
 *       lattices); the mass-median diameter is the smallest d at which fragments with diameter
 *       <= d hold at least half the total fragment volume.  A component is named by its smallest
 *       linear node index.
 *
 * Forward-mode tangent (complex step): compiled with ORC_COMPLEX_STEP the same source has
 * real = double _Complex and exports orc_cs_step and orc_cs_objective.  A parameter or state
 * perturbed by i h (h ~ 1e-30) gives dJ = Im J / h to rounding (Squire and Trapp, SIAM Rev.
 * 40, 1998): every operation of the step is complex-analytic except the comparisons (pivot
 * choice, the outflow clamp, the disc test), which act on real parts.
 *
 *   R12 Objectives of the adjoint (not in the paper), on the order parameter phi of a state's
 *       colour densities rho_k = sum_i S_i^k: the interface area sum of sqrt(|grad phi|^2 + eps^2)
 *       over 1 <= z <= nz-2 (isotropic stencil, x and y periodic), and the penetration length
 *       as a smooth maximum, delta log sum_n H(phi_n) exp(z_n / delta), with the redness weight
 *       H = ((1 + phi)/2)^2: 1 in pure red, 0 in pure blue (no tail that the exponential weight
 *       of distant blue nodes would amplify), smooth in between.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#ifdef ORC_COMPLEX_STEP
#include <complex.h>
typedef double _Complex real;
#define RE(x) creal(x)
#define SQRT(x) csqrt(x)
#define LOG(x) clog(x)
/* the complex build exports its own names */
#define orc_build_T orc_cs_build_T
#define orc_equilibrium orc_cs_equilibrium
#define orc_forcing_prime orc_cs_forcing_prime
#define orc_collide orc_cs_collide
#define orc_perturbation orc_cs_perturbation
#define orc_recolor orc_cs_recolor
#define orc_stream orc_cs_stream
#define orc_step orc_cs_step
#define orc_objective orc_cs_objective
double orc_inlet_xi(uint64_t seed, int64_t step, int32_t x, int32_t y, int32_t nx, int32_t ny);
#else
typedef double real;
#define RE(x) (x)
#define SQRT(x) sqrt(x)
#define LOG(x) log(x)
#endif
#define RABS(x) fabs(RE(x))

/* ---------------------------------------------------------------- lattice (Eq. (8)) */
static const int CX[27] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 1, -1, -1, 1};
static const int CY[27] = {0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 1, -1, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, -1, 1, 1, -1};
static const int CZ[27] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1, 1, -1, -1, 1, 1, -1, 1, -1};

enum { ORC_BC_PERIODIC = 0, ORC_BC_FREESLIP = 1, ORC_BC_INLET = 2, ORC_BC_CONVECTIVE = 3 };

typedef struct {
    int32_t nx, ny, nz;
    int32_t bc_zlo, bc_zhi;
    int32_t bc_x, bc_y;     /* PERIODIC or FREESLIP side walls (R14) */
} orc_grid;

typedef struct {
    real rho_r0, rho_b0;       /* initial densities rho_k^0 (Eq. (23)) */
    real nu_r, nu_b;           /* kinematic viscosities */
    real sigma;                /* interfacial tension */
    real beta;                 /* recolouring parameter */
    real g[3];                 /* gravity in F = (rho - rho_b^0) g */
    real s0, s1, s2b, s3, s4, s5, s6; /* relaxation rates of K (s_2nu follows from nu) */
    real u_in, d_in, noise_amp;/* inlet plug velocity, disc diameter, radial noise amplitude */
    uint64_t seed;               /* inlet noise seed */
    real eps_grad;             /* |grad phi| regulariser (R3) */
    real alpha_b;              /* 8/27 in the paper */
    real fourier[16];          /* inlet profile: a_1, b_1, ..., a_8, b_8 (R11) */
    int32_t alpha_mix;           /* 0: alpha-bar by (1 +- phi)/2 as printed; 1: by mass fraction (R15) */
} orc_params;

static double weight(int i) {
    int q = CX[i] * CX[i] + CY[i] * CY[i] + CZ[i] * CZ[i];
    if (q == 0) return 8.0 / 27.0;
    if (q == 1) return 2.0 / 27.0;
    if (q == 2) return 1.0 / 54.0;
    return 1.0 / 216.0;
}

/* Eq. (20) */
static real varphi(int i, real alpha) {
    int q = CX[i] * CX[i] + CY[i] * CY[i] + CZ[i] * CZ[i];
    if (q == 0) return alpha;
    if (q == 1) return 2.0 * (1.0 - alpha) / 19.0;
    if (q == 2) return (1.0 - alpha) / 38.0;
    return (1.0 - alpha) / 152.0;
}

/* Eq. (31) with c = 1 */
static double Bcoef(int i) {
    int q = CX[i] * CX[i] + CY[i] * CY[i] + CZ[i] * CZ[i];
    if (q == 0) return -10.0 / 27.0;
    if (q == 1) return 2.0 / 27.0;
    if (q == 2) return 1.0 / 54.0;
    return 1.0 / 216.0;
}

static int mirror_z(int i) {
    for (int j = 0; j < 27; ++j)
        if (CX[j] == CX[i] && CY[j] == CY[i] && CZ[j] == -CZ[i]) return j;
    return -1;
}

/* direction with velocity (cx, cy, cz) */
static int dir_of(int cx, int cy, int cz) {
    for (int j = 0; j < 27; ++j)
        if (CX[j] == cx && CY[j] == cy && CZ[j] == cz) return j;
    return -1;
}

/* Source column of a pull along c = (cxi, cyi) from column (x, y): wrapped where periodic,
 * reflected into the node's own layer at a free-slip side wall (R14), which reverses that
 * component of the direction leaving the source. */
static void side_source(const orc_grid *g, int x, int y, int *cxi, int *cyi, int *xs, int *ys) {
    *xs = x - *cxi;
    *ys = y - *cyi;
    if (*xs < 0 || *xs >= g->nx) {
        if (g->bc_x == ORC_BC_FREESLIP) { *xs = x; *cxi = -*cxi; }
        else *xs = ((*xs % g->nx) + g->nx) % g->nx;
    }
    if (*ys < 0 || *ys >= g->ny) {
        if (g->bc_y == ORC_BC_FREESLIP) { *ys = y; *cyi = -*cyi; }
        else *ys = ((*ys % g->ny) + g->ny) % g->ny;
    }
}

/* Neighbour column of (x, y) along (dx, dy) for gradient ghosts: wrapped where periodic,
 * the wall layer itself beyond a side wall (mirror ghost, R14). */
static void side_neighbour(const orc_grid *g, int x, int y, int dx, int dy, int *xn, int *yn) {
    *xn = x + dx;
    *yn = y + dy;
    if (*xn < 0 || *xn >= g->nx) *xn = g->bc_x == ORC_BC_FREESLIP ? x : ((*xn % g->nx) + g->nx) % g->nx;
    if (*yn < 0 || *yn >= g->ny) *yn = g->bc_y == ORC_BC_FREESLIP ? y : ((*yn % g->ny) + g->ny) % g->ny;
}

#ifndef ORC_COMPLEX_STEP
void orc_velocity_set(int32_t *c) {
    for (int i = 0; i < 27; ++i) {
        c[3 * i] = CX[i];
        c[3 * i + 1] = CY[i];
        c[3 * i + 2] = CZ[i];
    }
}

void orc_weights(double *w) {
    for (int i = 0; i < 27; ++i) w[i] = weight(i);
}

int orc_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

#endif

/* ---------------------------------------------------------- moment set (Eq. (14)) */
/* T[a][i]: row a is the a-th nonorthogonal central moment evaluated at direction i,
 * with cbar = c_i - u. */
void orc_build_T(const real *u, real *T) {
    for (int i = 0; i < 27; ++i) {
        real X = CX[i] - u[0], Y = CY[i] - u[1], Z = CZ[i] - u[2];
        real X2 = X * X, Y2 = Y * Y, Z2 = Z * Z;
        real r[27];
        r[0] = 1.0;
        r[1] = X;
        r[2] = Y;
        r[3] = Z;
        r[4] = X * Y;
        r[5] = X * Z;
        r[6] = Y * Z;
        r[7] = X2 - Y2;
        r[8] = X2 - Z2;
        r[9] = X2 + Y2 + Z2;
        r[10] = X * Y2 + X * Z2;
        r[11] = X2 * Y + Y * Z2;
        r[12] = X2 * Z + Y2 * Z;
        r[13] = X * Y2 - X * Z2;
        r[14] = X2 * Y - Y * Z2;
        r[15] = X2 * Z - Y2 * Z;
        r[16] = X * Y * Z;
        r[17] = X2 * Y2 + X2 * Z2 + Y2 * Z2;
        r[18] = X2 * Y2 + X2 * Z2 - Y2 * Z2;
        r[19] = X2 * Y2 - X2 * Z2;
        r[20] = X2 * Y * Z;
        r[21] = X * Y2 * Z;
        r[22] = X * Y * Z2;
        r[23] = X * Y2 * Z2;
        r[24] = X2 * Y * Z2;
        r[25] = X2 * Y2 * Z;
        r[26] = X2 * Y2 * Z2;
        for (int a = 0; a < 27; ++a) T[a * 27 + i] = r[a];
    }
}

/* Dense LU factorisation with partial pivoting (textbook Doolittle form), in place. */
static int lu_factor(real *A, int *piv) {
    for (int k = 0; k < 27; ++k) {
        int p = k;
        double best = RABS(A[k * 27 + k]);
        for (int r = k + 1; r < 27; ++r)
            if (RABS(A[r * 27 + k]) > best) { best = RABS(A[r * 27 + k]); p = r; }
        if (best == 0.0) return -1;
        piv[k] = p;
        if (p != k)
            for (int c = 0; c < 27; ++c) { real t = A[k * 27 + c]; A[k * 27 + c] = A[p * 27 + c]; A[p * 27 + c] = t; }
        for (int r = k + 1; r < 27; ++r) {
            A[r * 27 + k] /= A[k * 27 + k];
            for (int c = k + 1; c < 27; ++c) A[r * 27 + c] -= A[r * 27 + k] * A[k * 27 + c];
        }
    }
    return 0;
}

static void lu_solve(const real *LU, const int *piv, real *b) {
    for (int k = 0; k < 27; ++k)
        if (piv[k] != k) { real t = b[k]; b[k] = b[piv[k]]; b[piv[k]] = t; }
    for (int r = 0; r < 27; ++r)
        for (int c = 0; c < r; ++c) b[r] -= LU[r * 27 + c] * b[c];
    for (int r = 26; r >= 0; --r) {
        for (int c = r + 1; c < 27; ++c) b[r] -= LU[r * 27 + c] * b[c];
        b[r] /= LU[r * 27 + r];
    }
}

#ifndef ORC_COMPLEX_STEP
/* T(u)^-1 column by column (used by the tests against M^-1 N^-1 of Appendix A). */
int orc_T_inverse(const real *u, real *Tinv) {
    real T[729];
    int piv[27];
    orc_build_T(u, T);
    if (lu_factor(T, piv)) return -1;
    for (int j = 0; j < 27; ++j) {
        real e[27] = {0};
        e[j] = 1.0;
        lu_solve(T, piv, e);
        for (int r = 0; r < 27; ++r) Tinv[r * 27 + j] = e[r];
    }
    return 0;
}

#endif

/* K = diag(s0, s1 x3, s2nu x5, s2b, s3 x7, s4 x6, s5 x3, s6) */
static void relaxation_diag(const orc_params *p, real s2nu, real *K) {
    K[0] = p->s0;
    for (int a = 1; a <= 3; ++a) K[a] = p->s1;
    for (int a = 4; a <= 8; ++a) K[a] = s2nu;
    K[9] = p->s2b;
    for (int a = 10; a <= 16; ++a) K[a] = p->s3;
    for (int a = 17; a <= 22; ++a) K[a] = p->s4;
    for (int a = 23; a <= 25; ++a) K[a] = p->s5;
    K[26] = p->s6;
}

/* ------------------------------------------------------------ equilibrium (Eq. (18)) */
void orc_equilibrium(real rho, const real *u, real alpha, real nu, const real *grho, real *fe) {
    real G[3][3];
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) G[a][b] = (u[a] * grho[b] + u[b] * grho[a]) / 48.0;
    real usq = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    real ugr = u[0] * grho[0] + u[1] * grho[1] + u[2] * grho[2];
    for (int i = 0; i < 27; ++i) {
        real c[3] = {CX[i], CY[i], CZ[i]};
        real cu = c[0] * u[0] + c[1] * u[1] + c[2] * u[2];
        int q = CX[i] * CX[i] + CY[i] * CY[i] + CZ[i] * CZ[i];
        real poly = 3.0 * cu + 4.5 * cu * cu - 1.5 * usq + 4.5 * cu * cu * cu - 4.5 * cu * usq;
        real Gcc = 0.0;
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) Gcc += G[a][b] * c[a] * c[b];
        real Phi;
        if (q == 0) Phi = -3.0 * nu * ugr;
        else if (q == 1) Phi = 16.0 * nu * Gcc;
        else if (q == 2) Phi = 4.0 * nu * Gcc;
        else Phi = 1.0 * nu * Gcc;
        fe[i] = rho * (varphi(i, alpha) + weight(i) * poly) + Phi;
    }
}

/* ------------------------------------------------------------ forcing (Eq. (29)) */
void orc_forcing_prime(const real *u, const real *F, real *Fp) {
    for (int i = 0; i < 27; ++i) {
        real c[3] = {CX[i], CY[i], CZ[i]};
        real cu = c[0] * u[0] + c[1] * u[1] + c[2] * u[2];
        real s = 0.0;
        for (int a = 0; a < 3; ++a) s += (3.0 * (c[a] - u[a]) + 9.0 * cu * c[a]) * F[a];
        Fp[i] = weight(i) * s;
    }
}

/* ----------------------------------------- GMRT collision (Eqs. (11), (28)), literal */
/* Omega1 = -T^-1 K T (f - fe) + T^-1 (I - K/2) T F' with T = N M built from Eq. (14). */
int orc_collide(const real *f, const real *fe, const real *Fp, const real *u, const real *K, real *Omega1) {
    real T[729], LU[729];
    int piv[27];
    orc_build_T(u, T);
    memcpy(LU, T, sizeof(T));
    if (lu_factor(LU, piv)) return -1;
    real m[27], mf[27];
    for (int a = 0; a < 27; ++a) {
        real s = 0.0, sf = 0.0;
        for (int i = 0; i < 27; ++i) {
            s += T[a * 27 + i] * (f[i] - fe[i]);
            sf += T[a * 27 + i] * Fp[i];
        }
        m[a] = K[a] * s;                 /* K N M (f - fe) */
        mf[a] = (1.0 - 0.5 * K[a]) * sf; /* (I - K/2) N M F' */
    }
    lu_solve(LU, piv, m);  /* M^-1 N^-1 applied by solving T y = m */
    lu_solve(LU, piv, mf);
    for (int i = 0; i < 27; ++i) Omega1[i] = -m[i] + mf[i];
    return 0;
}

/* --------------------------------- perturbation (Eqs. (30), (31)), readings R1-R3 */
void orc_perturbation(real A, const real *gphi, real eps, real *Omega2) {
    real g2 = gphi[0] * gphi[0] + gphi[1] * gphi[1] + gphi[2] * gphi[2];
    real gmag = SQRT(g2 + eps * eps);
    for (int i = 0; i < 27; ++i) {
        real cg = CX[i] * gphi[0] + CY[i] * gphi[1] + CZ[i] * gphi[2];
        /* (A/2)|g| [w_i (c.g)^2/|g|^2 - B_i], written with one regularised |g| divisor */
        real one_colour = 0.5 * A * (weight(i) * cg * cg - Bcoef(i) * g2) / gmag;
        Omega2[i] = 0.0;
        for (int k = 0; k < 2; ++k) Omega2[i] += one_colour; /* R2: red and blue */
    }
}

/* ------------------------------------------------ recolouring (Eqs. (33), (34)) */
void orc_recolor(const real *fstar, real rho_r, real rho_b, real alpha_bar, real nu_bar,
                 real beta, const real *gphi, real eps, real *fr, real *fb) {
    real rho = rho_r + rho_b;
    real zero[3] = {0.0, 0.0, 0.0};
    real fe0[27];
    orc_equilibrium(rho, zero, alpha_bar, nu_bar, zero, fe0); /* f^(e)(rho, 0), R6 */
    real g2 = gphi[0] * gphi[0] + gphi[1] * gphi[1] + gphi[2] * gphi[2];
    real gmag = SQRT(g2 + eps * eps);
    for (int i = 0; i < 27; ++i) {
        double cnorm = sqrt((double)(CX[i] * CX[i] + CY[i] * CY[i] + CZ[i] * CZ[i]));
        real cos_t = 0.0;
        if (cnorm > 0.0) cos_t = (CX[i] * gphi[0] + CY[i] * gphi[1] + CZ[i] * gphi[2]) / (cnorm * gmag);
        real seg = beta * rho_r * rho_b / (rho * rho) * cos_t * fe0[i];
        fr[i] = rho_r / rho * fstar[i] + seg;
        fb[i] = rho_b / rho * fstar[i] - seg;
    }
}

/* ------------------------------------------------------------------ inlet noise (R7) */
#ifndef ORC_COMPLEX_STEP
/* SplitMix64 (Steele, Lea and Flood, OOPSLA 2014): state increment 0x9E3779B97F4A7C15
 * followed by the published 64-bit finaliser. */
uint64_t orc_splitmix64(uint64_t state) {
    uint64_t z = state + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

/* xi in [-1, 1): hash of (seed, step, x, y), top 24 bits scaled exactly. */
double orc_inlet_xi(uint64_t seed, int64_t step, int32_t x, int32_t y, int32_t nx, int32_t ny) {
    uint64_t idx = ((uint64_t)step * (uint64_t)ny + (uint64_t)y) * (uint64_t)nx + (uint64_t)x;
    uint64_t h = orc_splitmix64(seed ^ orc_splitmix64(idx));
    return (double)(h >> 40) * (1.0 / 8388608.0) - 1.0;
}

#endif

static int in_disc(const orc_grid *g, const orc_params *p, int x, int y) {
    double dx = 2.0 * x - (g->nx - 1), dy = 2.0 * y - (g->ny - 1);
    return dx * dx + dy * dy < RE(p->d_in) * RE(p->d_in);
}

static void inlet_velocity(const orc_grid *g, const orc_params *p, int64_t step, int x, int y, real *u) {
    double rx = x - 0.5 * (g->nx - 1), ry = y - 0.5 * (g->ny - 1);
    double r = sqrt(rx * rx + ry * ry);
    double xi = orc_inlet_xi(p->seed, step, x, y, g->nx, g->ny);
    real a = p->noise_amp * p->u_in * xi;
    u[0] = r > 0.0 ? a * rx / r : 0.0;
    u[1] = r > 0.0 ? a * ry / r : 0.0;
    double theta = atan2(ry, rx);
    real prof = 1.0;
    for (int m = 1; m <= 8; ++m)
        prof += p->fourier[2 * (m - 1)] * cos(m * theta) + p->fourier[2 * m - 1] * sin(m * theta);
    u[2] = p->u_in * prof;
}

static real alpha_red(const orc_params *p) {
    /* gamma = rho_r0/rho_b0 = (1 - alpha_b)/(1 - alpha_r) */
    real gamma = p->rho_r0 / p->rho_b0;
    return 1.0 - (1.0 - p->alpha_b) / gamma;
}

/* ----------------------------------------------------------------- indexing helpers */
static inline size_t nidx(const orc_grid *g, int x, int y, int z) {
    return ((size_t)z * g->ny + y) * g->nx + x;
}
static inline size_t pidx(const orc_grid *g, int k, int i, size_t n) {
    size_t N = (size_t)g->nx * g->ny * g->nz;
    return ((size_t)k * 27 + i) * N + n;
}
static inline int wrap(int a, int n) { return ((a % n) + n) % n; }

/* --------------------------------------------------------- streaming (Eq. (9), pull) */
/* f[k][i](x) = S[k][i](x - c_i) with the boundary rules R7, R8.  `hist` holds the
 * post-stream populations of the outflow plane at the previous step; on return
 * `hist_out` holds those of this step. */
void orc_stream(const orc_grid *g, const orc_params *p, const real *S, const real *hist,
                int64_t step, real *f, real *hist_out) {
    const int nx = g->nx, ny = g->ny, nz = g->nz, N = nz - 1;
    real alpha_r = alpha_red(p);
#pragma omp parallel for collapse(2) schedule(static)
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x)
                for (int i = 0; i < 27; ++i) {
                    int cxi = CX[i], cyi = CY[i], xs, ys, zs = z - CZ[i];
                    side_source(g, x, y, &cxi, &cyi, &xs, &ys);
                    const int ii = dir_of(cxi, cyi, CZ[i]); /* direction leaving the source (R14) */
                    size_t n = nidx(g, x, y, z);
                    for (int k = 0; k < 2; ++k) {
                        real v;
                        if (g->bc_zlo == ORC_BC_PERIODIC) {
                            v = S[pidx(g, k, ii, nidx(g, xs, ys, wrap(zs, nz)))];
                        } else if (zs < 0) {
                            if (g->bc_zlo == ORC_BC_INLET && in_disc(g, p, xs, ys)) {
                                if (k == 0) {
                                    real uin[3], fe[27], zero[3] = {0, 0, 0};
                                    inlet_velocity(g, p, step, xs, ys, uin);
                                    orc_equilibrium(p->rho_r0, uin, alpha_r, p->nu_r, zero, fe);
                                    v = fe[ii];
                                } else {
                                    v = 0.0;
                                }
                            } else {
                                v = S[pidx(g, k, mirror_z(ii), nidx(g, xs, ys, 0))];
                            }
                        } else if (zs > N) {
                            /* only free-slip reaches here; the convective plane is replaced below */
                            v = S[pidx(g, k, mirror_z(ii), nidx(g, xs, ys, N))];
                        } else {
                            v = S[pidx(g, k, ii, nidx(g, xs, ys, zs))];
                        }
                        f[pidx(g, k, i, n)] = v;
                    }
                }
    if (g->bc_zhi == ORC_BC_CONVECTIVE) {
#pragma omp parallel for schedule(static)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                size_t m = nidx(g, x, y, N - 1), n = nidx(g, x, y, N);
                /* u_z at N-1 after streaming (Eq. (13) with F = (rho - rho_b0) g) */
                real rho = 0.0, jz = 0.0;
                for (int k = 0; k < 2; ++k)
                    for (int i = 0; i < 27; ++i) {
                        rho += f[pidx(g, k, i, m)];
                        jz += f[pidx(g, k, i, m)] * CZ[i];
                    }
                real Fz = (rho - p->rho_b0) * p->g[2];
                real lam = (jz + 0.5 * Fz) / rho;
                if (RE(lam) < 0.0) lam = 0.0;
                if (RE(lam) > 1.0) lam = 1.0;
                for (int k = 0; k < 2; ++k)
                    for (int i = 0; i < 27; ++i) {
                        size_t h = ((size_t)(k * 27 + i) * ny + y) * nx + x;
                        real v = (hist[h] + lam * f[pidx(g, k, i, m)]) / (1.0 + lam);
                        f[pidx(g, k, i, n)] = v;
                        hist_out[h] = v;
                    }
            }
    }
}

/* --------------------------------------------------- one full step (Sections II, IV.A) */
/* S_in: post-collision state at step `step`; S_out: post-collision state at step+1.
 * mask (optional, nx*ny*nz bytes): nodes whose collision is evaluated; others get 0.
 * hist / hist_out: [2][27][ny][nx] outflow history (only read with a convective z_hi). */
int orc_step(const orc_grid *g, const orc_params *p, const real *S_in, const real *hist,
             int64_t step, real *S_out, real *hist_out, const uint8_t *mask) {
    const int nx = g->nx, ny = g->ny, nz = g->nz, N = nz - 1;
    const size_t nn = (size_t)nx * ny * nz;
    real *f = (real *)malloc(sizeof(real) * 54 * nn);
    real *rr = (real *)malloc(sizeof(real) * nn);
    real *rb = (real *)malloc(sizeof(real) * nn);
    if (!f || !rr || !rb) { free(f); free(rr); free(rb); return -2; }
    orc_stream(g, p, S_in, hist, step, f, hist_out);
    /* densities rho_k = sum_i f_i^k */
#pragma omp parallel for schedule(static)
    for (size_t n = 0; n < nn; ++n) {
        real a = 0.0, b = 0.0;
        for (int i = 0; i < 27; ++i) { a += f[pidx(g, 0, i, n)]; b += f[pidx(g, 1, i, n)]; }
        rr[n] = a;
        rb[n] = b;
    }
    const real alpha_b = p->alpha_b, alpha_r = alpha_red(p);
    int fail = 0;
#pragma omp parallel for collapse(2) schedule(dynamic, 1) reduction(| : fail)
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                size_t n = nidx(g, x, y, z);
                if (mask && !mask[n]) {
                    for (int k = 0; k < 2; ++k)
                        for (int i = 0; i < 27; ++i) S_out[pidx(g, k, i, n)] = 0.0;
                    continue;
                }
                /* isotropic gradients of phi and rho with the ghost rules R9 */
                real gphi[3] = {0, 0, 0}, grho[3] = {0, 0, 0};
                for (int j = 0; j < 27; ++j) {
                    int xn, yn, zn = z + CZ[j];
                    side_neighbour(g, x, y, CX[j], CY[j], &xn, &yn);
                    real a, b;
                    if (g->bc_zlo == ORC_BC_PERIODIC) {
                        size_t m = nidx(g, xn, yn, wrap(zn, nz));
                        a = rr[m]; b = rb[m];
                    } else if (zn < 0) {
                        if (g->bc_zlo == ORC_BC_INLET && in_disc(g, p, xn, yn)) {
                            a = p->rho_r0; b = 0.0;
                        } else {
                            size_t m = nidx(g, xn, yn, 0);
                            a = rr[m]; b = rb[m];
                        }
                    } else if (zn > N) {
                        size_t m = nidx(g, xn, yn, N);
                        a = rr[m]; b = rb[m];
                    } else {
                        size_t m = nidx(g, xn, yn, zn);
                        a = rr[m]; b = rb[m];
                    }
                    real phi_j = (a / p->rho_r0 - b / p->rho_b0) / (a / p->rho_r0 + b / p->rho_b0);
                    real rho_j = a + b;
                    real w = weight(j);
                    real c[3] = {CX[j], CY[j], CZ[j]};
                    for (int d = 0; d < 3; ++d) {
                        gphi[d] += 3.0 * w * phi_j * c[d];
                        grho[d] += 3.0 * w * rho_j * c[d];
                    }
                }
                /* colour-blind populations, densities, order parameter */
                real fb_[27];
                for (int i = 0; i < 27; ++i) fb_[i] = f[pidx(g, 0, i, n)] + f[pidx(g, 1, i, n)];
                real rho_r = rr[n], rho_b = rb[n], rho = rho_r + rho_b;
                real phi = (rho_r / p->rho_r0 - rho_b / p->rho_b0) / (rho_r / p->rho_r0 + rho_b / p->rho_b0);
                /* body force (Eq. (48)) and Guo velocity (Eq. (13)) */
                real F[3], u[3];
                for (int d = 0; d < 3; ++d) F[d] = (rho - p->rho_b0) * p->g[d];
                for (int d = 0; d < 3; ++d) {
                    real s = 0.0;
                    for (int i = 0; i < 27; ++i) s += fb_[i] * (d == 0 ? CX[i] : d == 1 ? CY[i] : CZ[i]);
                    u[d] = (s + 0.5 * F[d]) / rho;
                }
                /* mixture parameters */
                real alpha_bar = p->alpha_mix ? (rho_r * alpha_r + rho_b * alpha_b) / rho
                                              : 0.5 * (1.0 + phi) * alpha_r + 0.5 * (1.0 - phi) * alpha_b;
                real nu_bar = 1.0 / (0.5 * (1.0 + phi) / p->nu_r + 0.5 * (1.0 - phi) / p->nu_b);
                real s2nu = 1.0 / (3.0 * nu_bar + 0.5); /* Eq. (16) with c = dt = 1 */
                real tau = 1.0 / s2nu;
                real A = 9.0 * p->sigma / (4.0 * tau); /* Eq. (32), R4 */
                real K[27], fe[27], Fp[27], Om1[27], Om2[27], fs[27];
                relaxation_diag(p, s2nu, K);
                orc_equilibrium(rho, u, alpha_bar, nu_bar, grho, fe);
                orc_forcing_prime(u, F, Fp);
                if (orc_collide(fb_, fe, Fp, u, K, Om1)) { fail |= 1; continue; }
                orc_perturbation(A, gphi, p->eps_grad, Om2);
                for (int i = 0; i < 27; ++i) fs[i] = fb_[i] + Om1[i] + Om2[i];
                real fr[27], fbl[27];
                orc_recolor(fs, rho_r, rho_b, alpha_bar, nu_bar, p->beta, gphi, p->eps_grad, fr, fbl);
                for (int i = 0; i < 27; ++i) {
                    S_out[pidx(g, 0, i, n)] = fr[i];
                    S_out[pidx(g, 1, i, n)] = fbl[i];
                }
            }
    free(f); free(rr); free(rb);
    return fail ? -1 : 0;
}

#ifndef ORC_COMPLEX_STEP
/* --------------------------------------------------------- initial states (R10, Sec. III) */
/* Populations from fields rho_r, rho_b (nn each) and u (3*nn, component-major). */
void orc_init_fields(const orc_grid *g, const orc_params *p, const real *rho_r, const real *rho_b,
                     const real *u, real *S, real *hist) {
    const size_t nn = (size_t)g->nx * g->ny * g->nz;
    real alpha_r = alpha_red(p);
    for (size_t n = 0; n < nn; ++n) {
        real uu[3] = {u[n], u[nn + n], u[2 * nn + n]};
        real usq = uu[0] * uu[0] + uu[1] * uu[1] + uu[2] * uu[2];
        for (int i = 0; i < 27; ++i) {
            real cu = CX[i] * uu[0] + CY[i] * uu[1] + CZ[i] * uu[2];
            real poly = 3.0 * cu + 4.5 * cu * cu - 1.5 * usq + 4.5 * cu * cu * cu - 4.5 * cu * usq;
            S[pidx(g, 0, i, n)] = rho_r[n] * (varphi(i, alpha_r) + weight(i) * poly);
            S[pidx(g, 1, i, n)] = rho_b[n] * (varphi(i, p->alpha_b) + weight(i) * poly);
        }
    }
    /* history plane starts as the initial outflow-plane populations */
    const int N = g->nz - 1;
    for (int k = 0; k < 2; ++k)
        for (int i = 0; i < 27; ++i)
            for (int y = 0; y < g->ny; ++y)
                for (int x = 0; x < g->nx; ++x)
                    hist[((size_t)(k * 27 + i) * g->ny + y) * g->nx + x] = S[pidx(g, k, i, nidx(g, x, y, N))];
}

/* Static droplet of Section III: tanh profiles of width W around radius R, centre at
 * the domain centre ((n - 1)/2 in each direction), at rest. */
void orc_droplet_fields(const orc_grid *g, const orc_params *p, real R, real W, real *rho_r, real *rho_b) {
    real xc = 0.5 * (g->nx - 1), yc = 0.5 * (g->ny - 1), zc = 0.5 * (g->nz - 1);
    for (int z = 0; z < g->nz; ++z)
        for (int y = 0; y < g->ny; ++y)
            for (int x = 0; x < g->nx; ++x) {
                real r = sqrt((x - xc) * (x - xc) + (y - yc) * (y - yc) + (z - zc) * (z - zc));
                real t = tanh(2.0 * (r - R) / W);
                size_t n = nidx(g, x, y, z);
                rho_r[n] = 0.5 * p->rho_r0 * (1.0 - t);
                rho_b[n] = 0.5 * p->rho_b0 * (1.0 + t);
            }
}

/* --------------------------------------------------------------------- diagnostics */
/* Fields of a post-collision state: rho_k = sum_i S_i^k; rho u = sum_i S_i c_i - F/2
 * (the collision adds F to the momentum, Eqs. (11) and (28)); p from Eq. (26)
 * with rho and alpha-bar. */
void orc_fields(const orc_grid *g, const orc_params *p, const real *S, real *rho_r, real *rho_b,
                real *u, real *phi, real *pres) {
    const size_t nn = (size_t)g->nx * g->ny * g->nz;
    real alpha_r = alpha_red(p);
#pragma omp parallel for schedule(static)
    for (size_t n = 0; n < nn; ++n) {
        real a = 0.0, b = 0.0, j[3] = {0, 0, 0};
        for (int i = 0; i < 27; ++i) {
            real fr = S[pidx(g, 0, i, n)], fb = S[pidx(g, 1, i, n)];
            a += fr;
            b += fb;
            j[0] += (fr + fb) * CX[i];
            j[1] += (fr + fb) * CY[i];
            j[2] += (fr + fb) * CZ[i];
        }
        real rho = a + b;
        real ph = (a / p->rho_r0 - b / p->rho_b0) / (a / p->rho_r0 + b / p->rho_b0);
        for (int d = 0; d < 3; ++d) u[d * nn + n] = (j[d] - 0.5 * (rho - p->rho_b0) * p->g[d]) / rho;
        real alpha_bar = p->alpha_mix ? (a * alpha_r + b * p->alpha_b) / rho
                                      : 0.5 * (1.0 + ph) * alpha_r + 0.5 * (1.0 - ph) * p->alpha_b;
        rho_r[n] = a;
        rho_b[n] = b;
        phi[n] = ph;
        pres[n] = rho * 9.0 * (1.0 - alpha_bar) / 19.0;
    }
}

/* Per-colour total mass of a state (Neumaier-compensated sum in index order). */
void orc_mass(const orc_grid *g, const real *S, real *out) {
    const size_t nn = (size_t)g->nx * g->ny * g->nz;
    for (int k = 0; k < 2; ++k) {
        real s = 0.0, c = 0.0;
        for (int i = 0; i < 27; ++i)
            for (size_t n = 0; n < nn; ++n) {
                real v = S[pidx(g, k, i, n)], t = s + v;
                c += fabs(s) >= fabs(v) ? (s - t) + v : (v - t) + s;
                s = t;
            }
        out[k] = s + c;
    }
}

#endif

/* ------------------------------------------------------ adjoint objectives (R12) */
real orc_objective(const orc_grid *g, const orc_params *p, const real *S, int kind, const double *args) {
    const int nx = g->nx, ny = g->ny, nz = g->nz;
    const size_t nn = (size_t)nx * ny * nz;
    real *phi = (real *)malloc(sizeof(real) * nn);
    if (!phi) return (real)NAN;
    for (size_t n = 0; n < nn; ++n) {
        real a = 0.0, b = 0.0;
        for (int i = 0; i < 27; ++i) { a += S[pidx(g, 0, i, n)]; b += S[pidx(g, 1, i, n)]; }
        phi[n] = (a / p->rho_r0 - b / p->rho_b0) / (a / p->rho_r0 + b / p->rho_b0);
    }
    real J = 0.0;
    if (kind == 0) {
        double eps = args[0];
        for (int z = 1; z <= nz - 2; ++z)
            for (int y = 0; y < ny; ++y)
                for (int x = 0; x < nx; ++x) {
                    real gr[3] = {0, 0, 0};
                    for (int j = 0; j < 27; ++j) {
                        int xn, yn;
                        side_neighbour(g, x, y, CX[j], CY[j], &xn, &yn);
                        real v = phi[nidx(g, xn, yn, z + CZ[j])];
                        gr[0] += 3.0 * weight(j) * CX[j] * v;
                        gr[1] += 3.0 * weight(j) * CY[j] * v;
                        gr[2] += 3.0 * weight(j) * CZ[j] * v;
                    }
                    J += SQRT(gr[0] * gr[0] + gr[1] * gr[1] + gr[2] * gr[2] + eps * eps);
                }
    } else {
        double delta = args[0], N = nz - 1;
        real sum = 0.0;
        for (int z = 0; z < nz; ++z)
            for (int y = 0; y < ny; ++y)
                for (int x = 0; x < nx; ++x) {
                    real h = 0.5 * (1.0 + phi[nidx(g, x, y, z)]), H = h * h;
                    sum += H * exp((z - N) / delta);
                }
        J = N + delta * LOG(sum);
    }
    free(phi);
    return J;
}

#ifndef ORC_COMPLEX_STEP
/* ------------------------------------------------------------- fragments (R13) */
/* Breadth-first flood fill from every unvisited jet node in index order: the first node of a
 * component met in that scan is its smallest index, which names it.  Writes up to cap
 * (root, volume, touches z = 0) triples; returns the number of components or -2 on memory
 * exhaustion. */
int64_t orc_fragments(const orc_grid *g, const orc_params *p, const double *S, int connectivity, int64_t *roots,
                      int64_t *volumes, uint8_t *touch_z0, int64_t cap) {
    const int nx = g->nx, ny = g->ny, nz = g->nz;
    const size_t nn = (size_t)nx * ny * nz;
    const int pz = g->bc_zlo == ORC_BC_PERIODIC;
    uint8_t *jet = (uint8_t *)malloc(nn), *seen = (uint8_t *)calloc(nn, 1);
    int64_t *queue = (int64_t *)malloc(sizeof(int64_t) * nn);
    if (!jet || !seen || !queue) { free(jet); free(seen); free(queue); return -2; }
    for (size_t n = 0; n < nn; ++n) {
        double a = 0.0, b = 0.0;
        for (int i = 0; i < 27; ++i) { a += S[pidx(g, 0, i, n)]; b += S[pidx(g, 1, i, n)]; }
        double phi = (a / p->rho_r0 - b / p->rho_b0) / (a / p->rho_r0 + b / p->rho_b0);
        jet[n] = phi > 0.0;
    }
    int64_t count = 0;
    for (size_t s0 = 0; s0 < nn; ++s0) {
        if (!jet[s0] || seen[s0]) continue;
        size_t head = 0, tail = 0;
        queue[tail++] = (int64_t)s0;
        seen[s0] = 1;
        int64_t vol = 0;
        int touch = 0;
        while (head < tail) {
            int64_t n = queue[head++];
            ++vol;
            int x = (int)(n % nx), y = (int)((n / nx) % ny), z = (int)(n / ((int64_t)nx * ny));
            if (z == 0) touch = 1;
            for (int dz = -1; dz <= 1; ++dz)
                for (int dy = -1; dy <= 1; ++dy)
                    for (int dx = -1; dx <= 1; ++dx) {
                        int m = abs(dx) + abs(dy) + abs(dz);
                        if (m == 0 || (connectivity == 6 && m != 1)) continue;
                        int zz = z + dz, xx = x + dx, yy = y + dy;
                        if (pz) zz = wrap(zz, nz);
                        else if (zz < 0 || zz >= nz) continue;
                        if (xx < 0 || xx >= nx) {
                            if (g->bc_x == ORC_BC_FREESLIP) continue;
                            xx = wrap(xx, nx);
                        }
                        if (yy < 0 || yy >= ny) {
                            if (g->bc_y == ORC_BC_FREESLIP) continue;
                            yy = wrap(yy, ny);
                        }
                        size_t q = nidx(g, xx, yy, zz);
                        if (jet[q] && !seen[q]) { seen[q] = 1; queue[tail++] = (int64_t)q; }
                    }
        }
        if (count < cap) {
            if (roots) roots[count] = (int64_t)s0;
            if (volumes) volumes[count] = vol;
            if (touch_z0) touch_z0[count] = (uint8_t)touch;
        }
        ++count;
    }
    free(jet); free(seen); free(queue);
    return count;
}
#endif

#ifdef ORC_COMPLEX_STEP
/* The complex objective as (real part, imaginary part) through a pointer (a complex return
 * value does not cross every foreign-function interface). */
void orc_cs_objective_parts(const orc_grid *g, const orc_params *p, const real *S, int kind, const double *args,
                            double *out) {
    real J = orc_objective(g, p, S, kind, args);
    out[0] = creal(J);
    out[1] = cimag(J);
}
#endif
