/*
 * FP64 direct-sum visibility oracle.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call, link or
 * load this file; it exists so that tests, the smoke check and the CPU
 * baseline of the benchmark can compare the CUDA path against the plain
 * definition of the result.  It shares no code, header, table or constant
 * with the CUDA path.
 *
 * What it computes (paper Section 2.1):
 *   V^{pq}_{ij}(nu, t) = sum over sources n above the horizon of
 *       [ J(s_n, nu) C_n(nu) J(s_n, nu)^dagger ]_{pq}
 *       * exp(-2 pi i nu (x_i - x_j) . s_n(t) / c)
 * which is the RIME of Eq. (1) under the point-source approximation of
 * Eq. (3), with the coherency matrix of Eq. (2).  For an unpolarised sky the
 * single product is B(s_n, nu) I_n(nu) with the power beam B = |A|^2.
 *
 * Two evaluation modes:
 *   ORACLE_LITERAL  one sincos per (baseline, source);
 *   ORACLE_FACTORED per-antenna phasors F_an = exp(-2 pi i nu x_a . s_n / c)
 *                   and V_ij = sum_n c_n F_in conj(F_jn), the exact
 *                   factorisation of the fringe term written in Section 5.1
 *                   (review of the matrix-based algorithm).
 *
 * Conventions that the paper leaves open (each is stated, not derived):
 *  - baseline b_ij = x_i - x_j (the factorisation of Section 5.1 implies it);
 *  - sources contribute only when strictly above the horizon (Section 2.1);
 *  - the topocentric frame is East-North-Up, reached from equatorial unit
 *    vectors by the rigid rotation fixed by local sidereal time and latitude
 *    (Section 2.3, hybrid method, rigid-rotation part);
 *  - beams: Gaussian power beam exp(-4 ln2 theta^2 / FWHM(nu)^2) with
 *    FWHM(nu) = FWHM_ref * nu_ref / nu; Airy voltage 2 J1(x)/x with
 *    x = pi D nu sin(theta) / c; a uniform beam (A = 1) for analytic tests.
 *    The Jones matrix is A(theta) [[cos az, -sin az], [sin az, cos az]] with
 *    az measured east of north;
 *  - coherency C = [[I+Q, U+iV], [U-iV, I-Q]] exactly as printed in Eq. (2);
 *  - per-antenna beams (Section 2.2.3, Eq. 1 with A_i != A_j): antenna a has
 *    J_a = A_{b(a)}(theta) R(az), so the product of baseline (i, j) is
 *    J_i C J_j^dagger = A_{b(i)} A_{b(j)} R C R^dagger; evaluated as the
 *    unit-beam strengths times the two voltages, per baseline (literal) or
 *    folded into the antenna phasors (factored);
 *  - gridded (numerical) beams (Section 2.4): voltage samples per channel on
 *    a regular grid of zenith angle (zenith to horizon) and azimuth (east of
 *    north, periodic), interpolated bilinearly or by bicubic B-splines (the
 *    zenith-angle axis mirrored at its ends); they enter as per-antenna
 *    beams (one gridded beam for every antenna is the shared-beam case).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORACLE_C_LIGHT 299792458.0
#define ORACLE_LITERAL 0
#define ORACLE_FACTORED 1

#define ORACLE_BEAM_GAUSS 0
#define ORACLE_BEAM_AIRY 1
#define ORACLE_BEAM_UNIFORM 2
#define ORACLE_BEAM_GRID 3

typedef struct {
    int n_ant;
    const double *ant_enu;   /* [n_ant][3] metres, East North Up */
    int n_bl;
    const int *pairs;        /* [n_bl][2] antenna indices (i, j) */
    long n_src;
    const double *ra;        /* [n_src] rad */
    const double *dec;       /* [n_src] rad */
    int n_stokes;            /* 1 (I) or 4 (I, Q, U, V) */
    const double *flux;      /* [n_stokes][n_src][n_freq] Jy */
    int n_freq;
    const double *freq_hz;   /* [n_freq] */
    int n_time;
    const double *lst_rad;   /* [n_time] */
    double latitude_rad;
    int beam_kind;
    double beam_param[3];    /* GAUSS: fwhm_rad at ref, ref_hz; AIRY: dish diameter m */
    int polarized;           /* 0: one product (B I); 1: four products pq = 00, 01, 10, 11 */
    /* per-antenna beams (Section 2.2.3): antenna a has beam beam_of_ant[a] of the n_beams beams
     * (beam_kinds[k], beam_params[3k..3k+2]); beam_of_ant == NULL: every antenna has beam_kind. */
    int n_beams;
    const int *beam_kinds;
    const double *beam_params;
    const int *beam_of_ant;
    /* gridded beams (Section 2.4, numerical beams): beam k of kind ORACLE_BEAM_GRID has voltage samples
     * beam_grids[((k * n_freq + f) * grid_n_theta + i) * grid_n_phi + j] at zenith angle
     * i (pi/2) / (grid_n_theta - 1) and azimuth j 2 pi / grid_n_phi (east of north), channel f */
    int grid_n_theta, grid_n_phi;
    const double *beam_grids;
    /* 1: bilinear in the samples; 3: bicubic B-spline, beam_grids then holding the B-spline
     * coefficients of each plane (oracle.py computes them from the samples) */
    int grid_order;
} oracle_problem;

/* Equatorial (ra, dec) to topocentric East-North-Up unit vector at local
 * sidereal time lst and latitude lat: hour angle H = lst - ra, then
 *   E = -cos(dec) sin(H)
 *   N =  sin(dec) cos(lat) - cos(dec) cos(H) sin(lat)
 *   U =  sin(dec) sin(lat) + cos(dec) cos(H) cos(lat)       (Section 2.3) */
void oracle_enu(double ra, double dec, double lst, double lat, double *out3)
{
    double H = lst - ra;
    double cd = cos(dec), sd = sin(dec);
    double ch = cos(H), sh = sin(H);
    double cl = cos(lat), sl = sin(lat);
    out3[0] = -cd * sh;
    out3[1] = sd * cl - cd * ch * sl;
    out3[2] = sd * sl + cd * ch * cl;
}

/* Voltage of a gridded beam at zenith angle theta and azimuth az (east of north) by bilinear
 * interpolation (Section 2.4, numerical beams; bilinear is the lowest order the section names) in the
 * samples plane[i * n_phi + j] at theta_i = i (pi/2) / (n_theta - 1), az_j = j 2 pi / n_phi, the
 * azimuth periodic. */
double oracle_voltage_grid(const double *plane, int n_theta, int n_phi, double theta, double az)
{
    const double dth = (M_PI / 2.0) / (n_theta - 1), dph = 2.0 * M_PI / n_phi;
    double u = theta / dth;
    int i = (int)floor(u);
    if (i > n_theta - 2) i = n_theta - 2;
    if (i < 0) i = 0;
    const double a = u - i;
    double azw = fmod(az, 2.0 * M_PI);
    if (azw < 0.0) azw += 2.0 * M_PI;
    const double v = azw / dph;
    int j = (int)floor(v);
    const double b = v - j;
    const int j0 = ((j % n_phi) + n_phi) % n_phi, j1 = (j0 + 1) % n_phi;
    return (1.0 - a) * (1.0 - b) * plane[i * n_phi + j0] + (1.0 - a) * b * plane[i * n_phi + j1] +
           a * (1.0 - b) * plane[(i + 1) * n_phi + j0] + a * b * plane[(i + 1) * n_phi + j1];
}

/* Cubic B-spline B3 at offsets (a + 1, a, 1 - a, 2 - a) from the four nearest knots, a in [0, 1). */
static void bspline3_weights(double a, double w[4])
{
    const double b = 1.0 - a;
    w[0] = b * b * b / 6.0;
    w[1] = (3.0 * a * a * a - 6.0 * a * a + 4.0) / 6.0;
    w[2] = (3.0 * b * b * b - 6.0 * b * b + 4.0) / 6.0;
    w[3] = a * a * a / 6.0;
}

/* Voltage of a gridded beam by bicubic B-spline interpolation (Section 2.4 names bicubic among the
 * orders of its beam interpolation): coef[i * n_phi + j] are the B-spline coefficients of the plane
 * on the same grid as oracle_voltage_grid, the zenith-angle axis continued by mirror symmetry about
 * its first and last samples, the azimuth axis periodic. */
double oracle_voltage_grid3(const double *coef, int n_theta, int n_phi, double theta, double az)
{
    const double dth = (M_PI / 2.0) / (n_theta - 1), dph = 2.0 * M_PI / n_phi;
    const double u = theta / dth;
    int i = (int)floor(u);
    if (i > n_theta - 2) i = n_theta - 2;
    if (i < 0) i = 0;
    double azw = fmod(az, 2.0 * M_PI);
    if (azw < 0.0) azw += 2.0 * M_PI;
    const double v = azw / dph;
    const int j = (int)floor(v);
    double wt[4], wp[4];
    bspline3_weights(u - i, wt);
    bspline3_weights(v - j, wp);
    double acc = 0.0;
    for (int r = 0; r < 4; ++r) {
        int ii = i - 1 + r;
        if (ii < 0) ii = -ii;
        if (ii > n_theta - 1) ii = 2 * (n_theta - 1) - ii;
        for (int c = 0; c < 4; ++c) {
            const int jj = (((j - 1 + c) % n_phi) + n_phi) % n_phi;
            acc += wt[r] * wp[c] * coef[ii * n_phi + jj];
        }
    }
    return acc;
}

/* Scalar voltage response A(theta, nu) of the beam (Section 2.4, analytic beams). */
double oracle_voltage(int kind, const double *param, double theta, double nu)
{
    if (kind == ORACLE_BEAM_GAUSS) {
        double fwhm = param[0] * param[1] / nu;
        double power = exp(-4.0 * log(2.0) * theta * theta / (fwhm * fwhm));
        return sqrt(power);
    }
    if (kind == ORACLE_BEAM_AIRY) {
        double x = M_PI * param[0] * nu * sin(theta) / ORACLE_C_LIGHT;
        if (fabs(x) < 1e-8) return 1.0 - x * x / 8.0;
        return 2.0 * j1(x) / x;
    }
    return 1.0;
}

/* Source strengths for one source at topocentric direction s (up > 0):
 * c = J C J^dagger (Eq. 1-2), or B I for the unpolarised single product.
 * stokes[4] = I, Q, U, V.  out holds n_pol complex numbers as (re, im). */
void oracle_strength(int kind, const double *param, int polarized, const double *s,
                     double nu, const double *stokes, double *out)
{
    double theta = acos(s[2] > 1.0 ? 1.0 : s[2]);
    double A = oracle_voltage(kind, param, theta, nu);
    if (!polarized) {
        out[0] = A * A * stokes[0];
        out[1] = 0.0;
        return;
    }
    double az = atan2(s[0], s[1]);
    double ca = cos(az), sa = sin(az);
    /* J = A R, R = [[ca, -sa], [sa, ca]] (real) */
    double J[2][2] = {{A * ca, -A * sa}, {A * sa, A * ca}};
    double I = stokes[0], Q = stokes[1], U = stokes[2], V = stokes[3];
    /* C as (re, im) */
    double Cr[2][2] = {{I + Q, U}, {U, I - Q}};
    double Ci[2][2] = {{0.0, V}, {-V, 0.0}};
    /* T = J C */
    double Tr[2][2], Ti[2][2];
    for (int p = 0; p < 2; ++p)
        for (int q = 0; q < 2; ++q) {
            Tr[p][q] = J[p][0] * Cr[0][q] + J[p][1] * Cr[1][q];
            Ti[p][q] = J[p][0] * Ci[0][q] + J[p][1] * Ci[1][q];
        }
    /* (J C J^dagger)_{pq} = sum_k T_{pk} conj(J_{qk}); J real */
    for (int p = 0; p < 2; ++p)
        for (int q = 0; q < 2; ++q) {
            double re = Tr[p][0] * J[q][0] + Tr[p][1] * J[q][1];
            double im = Ti[p][0] * J[q][0] + Ti[p][1] * J[q][1];
            out[2 * (2 * p + q)] = re;
            out[2 * (2 * p + q) + 1] = im;
        }
}

static void stokes_of(const oracle_problem *P, long n, int f, double *st)
{
    for (int k = 0; k < 4; ++k) st[k] = 0.0;
    for (int k = 0; k < P->n_stokes && k < 4; ++k)
        st[k] = P->flux[((size_t)k * P->n_src + n) * P->n_freq + f];
}

/* Visibilities into vis[n_freq][n_time][n_bl][n_pol] as (re, im) doubles.
 * Returns 0 on success, nonzero on bad arguments or allocation failure. */
int oracle_vis(const oracle_problem *P, double *vis, int mode, int n_threads)
{
    if (!P || !vis || P->n_ant < 1 || P->n_bl < 0 || P->n_src < 0 || P->n_freq < 0 ||
        P->n_time < 0 || (P->n_stokes != 1 && P->n_stokes != 4))
        return 1;
    if (P->polarized && P->n_stokes != 4) return 1;
#ifdef _OPENMP
    if (n_threads > 0) omp_set_num_threads(n_threads);
#else
    (void)n_threads;
#endif
    const int n_pol = P->polarized ? 4 : 1;
    const long NS = P->n_src;
    const int multi = P->beam_of_ant != NULL && P->n_beams >= 1 && P->beam_kinds && P->beam_params;
    if (multi)
        for (int a = 0; a < P->n_ant; ++a)
            if (P->beam_of_ant[a] < 0 || P->beam_of_ant[a] >= P->n_beams) return 1;
    const int nbeam = multi ? P->n_beams : 1;
    double *volt = (double *)malloc(sizeof(double) * nbeam * (NS > 0 ? NS : 1));   /* [v][beam] */
    double *dir = (double *)malloc(sizeof(double) * 3 * (NS > 0 ? NS : 1));
    double *str = (double *)malloc(sizeof(double) * 2 * n_pol * (NS > 0 ? NS : 1));
    long *vis_idx = (long *)malloc(sizeof(long) * (NS > 0 ? NS : 1));
    const long BLK = 4096;
    double *F = NULL;
    if (mode == ORACLE_FACTORED)
        F = (double *)malloc(sizeof(double) * 2 * (size_t)P->n_ant * BLK);
    if (!dir || !str || !vis_idx || !volt || (mode == ORACLE_FACTORED && !F)) {
        free(dir); free(str); free(vis_idx); free(F); free(volt);
        return 2;
    }
    for (int t = 0; t < P->n_time; ++t) {
        /* topocentric directions at this time, horizon cut */
        long nv = 0;
        for (long n = 0; n < NS; ++n) {
            double s[3];
            oracle_enu(P->ra[n], P->dec[n], P->lst_rad[t], P->latitude_rad, s);
            if (s[2] > 0.0) {
                dir[3 * nv] = s[0]; dir[3 * nv + 1] = s[1]; dir[3 * nv + 2] = s[2];
                vis_idx[nv++] = n;
            }
        }
        for (int f = 0; f < P->n_freq; ++f) {
            const double nu = P->freq_hz[f];
            const double k0 = 2.0 * M_PI * nu / ORACLE_C_LIGHT;
#pragma omp parallel for schedule(static)
            for (long v = 0; v < nv; ++v) {
                double st[4];
                stokes_of(P, vis_idx[v], f, st);
                if (!multi) {
                    oracle_strength(P->beam_kind, P->beam_param, P->polarized, &dir[3 * v], nu, st,
                                    &str[2 * n_pol * v]);
                } else {
                    /* unit-beam strengths; the voltages of the antennas' beams multiply them per baseline */
                    double none[3] = {0.0, 0.0, 0.0};
                    oracle_strength(ORACLE_BEAM_UNIFORM, none, P->polarized, &dir[3 * v], nu, st,
                                    &str[2 * n_pol * v]);
                    double theta = acos(dir[3 * v + 2] > 1.0 ? 1.0 : dir[3 * v + 2]);
                    double az = atan2(dir[3 * v], dir[3 * v + 1]);
                    for (int k = 0; k < nbeam; ++k)
                        volt[(size_t)v * nbeam + k] =
                            P->beam_kinds[k] == ORACLE_BEAM_GRID
                                ? (P->grid_order == 3 ? oracle_voltage_grid3 : oracle_voltage_grid)(
                                      P->beam_grids + ((size_t)k * P->n_freq + f) * P->grid_n_theta * P->grid_n_phi,
                                      P->grid_n_theta, P->grid_n_phi, theta, az)
                                : oracle_voltage(P->beam_kinds[k], &P->beam_params[3 * k], theta, nu);
                }
            }
            double *out = vis + (((size_t)f * P->n_time + t) * P->n_bl) * n_pol * 2;
            if (mode == ORACLE_LITERAL) {
#pragma omp parallel for schedule(dynamic, 4)
                for (int b = 0; b < P->n_bl; ++b) {
                    const double *xi = &P->ant_enu[3 * P->pairs[2 * b]];
                    const double *xj = &P->ant_enu[3 * P->pairs[2 * b + 1]];
                    double bx = xi[0] - xj[0], by = xi[1] - xj[1], bz = xi[2] - xj[2];
                    const int bi = multi ? P->beam_of_ant[P->pairs[2 * b]] : 0;
                    const int bj = multi ? P->beam_of_ant[P->pairs[2 * b + 1]] : 0;
                    double acc[8] = {0};
                    for (long v = 0; v < nv; ++v) {
                        double ph = -k0 * (bx * dir[3 * v] + by * dir[3 * v + 1] + bz * dir[3 * v + 2]);
                        double g = multi ? volt[(size_t)v * nbeam + bi] * volt[(size_t)v * nbeam + bj] : 1.0;
                        double c = g * cos(ph), s = g * sin(ph);
                        for (int p = 0; p < n_pol; ++p) {
                            double sr = str[2 * (n_pol * v + p)], si = str[2 * (n_pol * v + p) + 1];
                            acc[2 * p] += sr * c - si * s;
                            acc[2 * p + 1] += sr * s + si * c;
                        }
                    }
                    for (int p = 0; p < 2 * n_pol; ++p) out[(size_t)b * n_pol * 2 + p] = acc[p];
                }
            } else {
                for (int b = 0; b < P->n_bl * n_pol * 2; ++b) out[b] = 0.0;
                for (long v0 = 0; v0 < nv; v0 += BLK) {
                    long nb = (nv - v0 < BLK) ? nv - v0 : BLK;
#pragma omp parallel for schedule(static)
                    for (int a = 0; a < P->n_ant; ++a) {
                        const double *xa = &P->ant_enu[3 * a];
                        for (long v = 0; v < nb; ++v) {
                            const double *s = &dir[3 * (v0 + v)];
                            double ph = -k0 * (xa[0] * s[0] + xa[1] * s[1] + xa[2] * s[2]);
                            double g = multi ? volt[(size_t)(v0 + v) * nbeam + P->beam_of_ant[a]] : 1.0;
                            F[2 * ((size_t)a * BLK + v)] = g * cos(ph);
                            F[2 * ((size_t)a * BLK + v) + 1] = g * sin(ph);
                        }
                    }
#pragma omp parallel for schedule(dynamic, 16)
                    for (int b = 0; b < P->n_bl; ++b) {
                        const double *Fi = &F[2 * (size_t)P->pairs[2 * b] * BLK];
                        const double *Fj = &F[2 * (size_t)P->pairs[2 * b + 1] * BLK];
                        double acc[8] = {0};
                        for (long v = 0; v < nb; ++v) {
                            /* e = F_i conj(F_j) */
                            double er = Fi[2 * v] * Fj[2 * v] + Fi[2 * v + 1] * Fj[2 * v + 1];
                            double ei = Fi[2 * v + 1] * Fj[2 * v] - Fi[2 * v] * Fj[2 * v + 1];
                            for (int p = 0; p < n_pol; ++p) {
                                double sr = str[2 * (n_pol * (v0 + v) + p)];
                                double si = str[2 * (n_pol * (v0 + v) + p) + 1];
                                acc[2 * p] += sr * er - si * ei;
                                acc[2 * p + 1] += sr * ei + si * er;
                            }
                        }
                        for (int p = 0; p < 2 * n_pol; ++p) out[(size_t)b * n_pol * 2 + p] += acc[p];
                    }
                }
            }
        }
    }
    free(dir); free(str); free(vis_idx); free(F); free(volt);
    return 0;
}

int oracle_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
