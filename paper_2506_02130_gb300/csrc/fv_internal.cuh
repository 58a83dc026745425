// Internal declarations shared by the translation units of libfftvis_gb300.
//
// Notation (Section 2.2, Eq. 4-5): sources s_n are topocentric direction
// cosines (E, N, U); targets x_k = -2 pi nu b_k / c; the result of one slice is
// f_k = sum_n c_n exp(i x_k . s_n).  The type-3 transform is evaluated as
//   f_k = e^{i x_k.C} * prod_i (4/w^2)/Phihat(a_ki)
//         * sum_m prod_i phi((2/w)(p_ki - m_i)) * P_m,
//   P_m = sum_l g_l prod_i [1/Phihat(l_i w pi / M_i)] e^{2 pi i l.m/M},
//   g_l = sum_n c_n e^{i D.(s_n - C)} prod_i phi((2/w)(l_i - q_ni)),
// with C, S the centre and half-extent of the sources, D, X those of the
// targets, q = (s - C) sigma X / pi the source grid coordinate (cells),
// p = (x - D) M / (2 sigma X) the target coordinate on the FFT grid of M
// points, a = (x - D) w pi / (2 sigma X), phi the ES kernel of Section 2.2
// (step 1) and Phihat(k) = int_{-1}^{1} phi(z) cos(k z) dz.  The grid size
// per dimension is nf1 >= 2 sigma X S / pi + w (Eq. 5).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <math.h>

#define FV_C_LIGHT 299792458.0
#define FV_MAX_STAGES 8
#define FV_ZDIRECT_MAX 16

namespace fv {

// aligned to its size, so that a complex value moves with one 8- or 16-byte load or store
template <class T> struct alignas(2 * sizeof(T)) cpx { T x, y; };

template <class T> __host__ __device__ __forceinline__ cpx<T> cmk(T a, T b) { cpx<T> r; r.x = a; r.y = b; return r; }
template <class T> __host__ __device__ __forceinline__ cpx<T> cadd(cpx<T> a, cpx<T> b) { return cmk<T>(a.x + b.x, a.y + b.y); }
template <class T> __host__ __device__ __forceinline__ cpx<T> csub(cpx<T> a, cpx<T> b) { return cmk<T>(a.x - b.x, a.y - b.y); }
template <class T> __host__ __device__ __forceinline__ cpx<T> cmul(cpx<T> a, cpx<T> b) {
    return cmk<T>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
template <class T> __host__ __device__ __forceinline__ cpx<T> cscale(cpx<T> a, T s) { return cmk<T>(a.x * s, a.y * s); }
// multiply by +i
template <class T> __host__ __device__ __forceinline__ cpx<T> cmuli(cpx<T> a) { return cmk<T>(-a.y, a.x); }

// Geometry of one dimension of one slice's transform.
struct DimGeom {
    int nf1;        // spreading grid points
    int M;          // FFT length (sigma * nf1, 2^a 3^b 5^c)
    int B;          // band of FFT outputs kept: indices m in [-H, B-1-H]
    int H;          // band offset
    double qscale;  // sigma X / pi : (s - C) -> source grid coordinate (cells)
    double pscale;  // M / (2 sigma X) : (x - D) -> target coordinate (FFT cells)
    double D;       // target centre (rad)
    double C;       // source centre
    int nstages;
    int radix[FV_MAX_STAGES];
    unsigned mr_mul[FV_MAX_STAGES], mr_sh[FV_MAX_STAGES];   // division by M / radix[s]
    unsigned ns_mul[FV_MAX_STAGES], ns_sh[FV_MAX_STAGES];   // division by prod(radix[0..s-1])
};

struct BeamParams {
    int kind;           // 0 gauss, 1 airy, 2 uniform, 3 gridded
    double p0, p1, p2;
    // the FP32 beam's constant, set on the host with the parameters (beam_float_constant): Gaussian
    // FWHM(nu) nu = p0 p1 (rad Hz); Airy pi D / c (the argument per Hz and per unit sin theta)
    float pf;
    // gridded beams (Section 2.4, numerical beams): voltage samples [n_freq][n_th][n_ph] on the grid
    // theta_i = i (pi/2) / (n_th - 1) (zenith angle), phi_j = j 2 pi / n_ph (azimuth east of north)
    const void *grid;   // device samples (order 1) or B-spline coefficients (order 3), FP64 if grid_fp64
    int grid_fp64, n_th, n_ph, grid_order;
};

// The FP32 beam constant of a beam, set on the host when its parameters are (Gaussian FWHM(nu) nu;
// Airy pi D / c; 0 otherwise).
inline void beam_float_constant(BeamParams &b)
{
    b.pf = b.kind == 0 ? (float)(b.p0 * b.p1) : (b.kind == 1 ? (float)(M_PI * b.p0 / FV_C_LIGHT) : 0.0f);
}

// Per-time binning geometry: bins are tiles of the top (highest-frequency)
// channel's grid in (x, y).
struct TimeBin {
    double R[9];            // equatorial -> ENU rotation at this time
    double C[3];            // source centre
    double qscale_top[3];   // grid scale of the top channel
    double D_top[3];        // target centre of the top channel (prephase D.(s - C))
    int d;                  // dimensions of the transform
    int nf1_top[3];
    int T[2];               // tile (= bin) size in cells
    int nbx, nby;           // bins per axis
};

#define FV_SPREAD_SMEM_MAX (96 * 1024)

// Everything a slice's kernels need, passed by value.
struct SliceGeom {
    double R[9];        // equatorial -> ENU rotation at this time (row major)
    double nu;          // Hz
    double kappa;       // 2 pi nu / c
    int d;              // 2 or 3
    int w;              // kernel width
    double beta;        // ES shape
    int n_pol;          // 1 or 4
    int polarized;
    int n_stokes;
    BeamParams beam;
    BeamParams beam2;   // per-antenna beams (Section 2.2.3): the second antenna's beam of the baseline
    int two_beams;      // 0: the product is beam x beam; 1: beam x beam2
    DimGeom dim[3];
    // x and y prescale tables 1/Phihat (grid precision) that the tiled spreading kernels apply when they
    // store each grid cell (the FFT passes then skip them); nullptr: the FFT passes apply them
    const void *pre_x, *pre_y;
    // kappa / kappa_top of this channel as a float pair (hi + lo): the FP32 grids scale the top channel's
    // per-time coordinates and prephase by it
    float rsc_hi, rsc_lo;
    // the plan's channel-major copy of the fluxes, [n_freq][n_src][n_stokes] (flux precision), or nullptr:
    // the caller's [n_stokes][n_src][n_freq]
    const void *flux_t;
    // Chebyshev height terms of a non-coplanar array on a two-dimensional grid (0: none): dim[2].nf1 = K
    // planes; a source's term argument is u = (n - hc) / hs (n its up component), a target's weights
    // follow from k b_up (height_weight)
    int K;
    double hc, hs;
    float hc_f, hs_inv_f;
    // nu and beta rounded to FP32 once on the host (a per-thread FP64 -> FP32 conversion runs on the
    // narrow FP64 pipe)
    float nu_f, beta_f;
    // FP32 two-dimensional interpolation without FP64: the target's grid coordinate is
    // p_i = -(kappa pscale_i) (b_i - bcen_i) and its postphase argument -kappa (b . C), formed as
    // double-float products of the per-channel factors (a_i = kappa pscale_i and kappa as float pairs)
    // and the per-target tables tgt_db[u] = (b_x - bcen_x, b_y - bcen_y) and tgt_bc[u] = b . C (float
    // pairs, channel independent; nullptr: the FP64 set-up)
    const float4 *tgt_db;
    const float2 *tgt_bc;
    float a_hi[2], a_lo[2], kap_hi, kap_lo;
};

template <class G> __device__ __forceinline__ G geom_nu(const SliceGeom &g);
template <> __device__ __forceinline__ double geom_nu<double>(const SliceGeom &g) { return g.nu; }
template <> __device__ __forceinline__ float geom_nu<float>(const SliceGeom &g) { return g.nu_f; }
template <class G> __device__ __forceinline__ G geom_beta(const SliceGeom &g);
template <> __device__ __forceinline__ double geom_beta<double>(const SliceGeom &g) { return g.beta; }
template <> __device__ __forceinline__ float geom_beta<float>(const SliceGeom &g) { return g.beta_f; }

// J_q(x) by its power series sum_m (-1)^m (x/2)^(2m+q) / (m! (m+q)!) (FP64; |x| is a few units at most here,
// so the terms fall fast and do not cancel badly)
__device__ __forceinline__ double bessel_jq(int q, double x, double rel_tol = 1e-18)
{
    const double h = 0.5 * x;
    double term = 1.0;
    for (int k = 1; k <= q; ++k) term *= h / k;
    double sum = term;
    const double h2 = h * h;
    for (int m = 1; m < 80; ++m) {
        term *= -h2 / ((double)m * (double)(m + q));
        sum += term;
        if (fabs(term) <= rel_tol * fabs(sum)) break;
    }
    return sum;
}

// Weight of height term q of the target with up baseline component b_up (m):
//   exp(-i k b_up hc) eps_q (-i)^q J_q(k b_up hs),  k = 2 pi nu / c,
// so that sum_q weight_q T_q((n - hc) / hs) = exp(-i k b_up n) (Jacobi-Anger).
template <class G>
__device__ __forceinline__ cpx<G> height_weight(const SliceGeom &g, double b_up, int q)
{
    const double a = g.kappa * b_up;
    if (sizeof(G) == 4 && fabs(a * g.hs) <= 2.0) {
        // FP32 grids, |a hs| <= 2: every term of the series is below the first, so FP32 arithmetic keeps
        // its 7 digits; the phase a hc is reduced to [-pi, pi] in FP64 first
        const float x = (float)(a * g.hs), h = 0.5f * x;
        float term = 1.0f;
        for (int k = 1; k <= q; ++k) term *= h / (float)k;
        float sum = term;
        const float h2 = h * h;
        for (int m = 1; m < 24; ++m) {
            term *= -h2 / ((float)m * (float)(m + q));
            sum += term;
            if (fabsf(term) <= 1e-8f * fabsf(sum)) break;
        }
        double ph = a * g.hc;
        ph -= 6.283185307179586476925 * rint(ph * 0.15915494309189533577);
        float sb, cb;
        sincosf((float)ph, &sb, &cb);
        const float j = (q == 0 ? 1.0f : 2.0f) * sum;
        float re = cb * j, im = -sb * j;
        for (int k = 0; k < (q & 3); ++k) {
            const float t = re;
            re = im;
            im = -t;
        }
        return cmk<G>((G)re, (G)im);
    }
    // FP32 grids keep about 7 digits: the series stops at 1e-10 relative there
    const double j = (q == 0 ? 1.0 : 2.0) * bessel_jq(q, a * g.hs, sizeof(G) == 4 ? 1e-10 : 1e-18);
    double sb, cb;
    sincos(a * g.hc, &sb, &cb);
    double re = cb * j, im = -sb * j;                  // exp(-i a hc) eps_q J_q
    for (int k = 0; k < (q & 3); ++k) {                // times (-i)^q
        const double t = re;
        re = im;
        im = -t;
    }
    return cmk<G>((G)re, (G)im);
}

// Position of Stokes parameter k of source n at channel f in the fluxes a slice reads (flux_index) and
// the array it is in: the channel-major copy when there is one (one channel's Stokes values of a
// source are adjacent), else the caller's layout.
__host__ __device__ __forceinline__ size_t flux_index(const SliceGeom &g, int k, long n, long n_src, int n_freq, int f)
{
    return g.flux_t ? ((size_t)f * n_src + n) * g.n_stokes + k : ((size_t)k * n_src + n) * n_freq + f;
}

// Beam voltage A(theta) of the analytic beams (Section 2.4): Gaussian power beam,
// Airy disc, or none.  rho = sin(zenith angle), s2 = cos(zenith angle).
template <class G> __device__ __forceinline__ G voltage(const BeamParams &b, G rho, G s2, G nu);
template <> __device__ __forceinline__ double voltage<double>(const BeamParams &b, double rho, double s2, double nu)
{
    if (b.kind == 0) {
        double theta = atan2(rho, s2);
        double fwhm = b.p0 * b.p1 / nu;
        return exp(-2.0 * M_LN2 * theta * theta / (fwhm * fwhm));
    }
    if (b.kind == 1) {
        double x = M_PI * b.p0 * nu * rho / FV_C_LIGHT;
        return x < 1e-8 ? 1.0 - 0.125 * x * x : 2.0 * j1(x) / x;
    }
    return 1.0;
}
// 2 J1(x) / x in FP32 for x >= 0 from the polynomial approximations of Abramowitz & Stegun (1964),
// 9.4.4 (|x| <= 3: error of J1(x)/x below 1.3e-8) and 9.4.6 (x >= 3: modulus and phase in 3/x, errors
// below 4e-8 and 9e-8), so that the FP32 beam needs no FP64 arithmetic
__device__ __forceinline__ float airy_2j1_over_x(float x)
{
    if (x <= 3.0f) {
        const float y = (x * (1.0f / 3.0f)) * (x * (1.0f / 3.0f));
        const float p = 0.5f + y * (-0.56249985f + y * (0.21093573f + y * (-0.03954289f + y * (0.00443319f +
                        y * (-0.00031761f + y * 0.00001109f)))));
        return 2.0f * p;
    }
    const float z = 3.0f / x;
    const float f1 = 0.79788456f + z * (0.00000156f + z * (0.01659667f + z * (0.00017105f + z * (-0.00249511f +
                     z * (0.00113653f + z * (-0.00020033f))))));
    const float th = x - 2.35619449f + z * (0.12499612f + z * (0.00005650f + z * (-0.00637879f + z * (0.00074348f +
                     z * (0.00079824f + z * (-0.00029166f))))));
    return 2.0f * f1 * cosf(th) / (x * sqrtf(x));
}

template <> __device__ __forceinline__ float voltage<float>(const BeamParams &b, float rho, float s2, float nu)
{
    if (b.kind == 0) {
        float theta = atan2f(rho, s2);
        float fwhm = b.pf / nu;
        return expf(-2.0f * 0.69314718055994531f * theta * theta / (fwhm * fwhm));
    }
    if (b.kind == 1) {
        float x = b.pf * nu * rho;
        return airy_2j1_over_x(x);
    }
    return 1.0f;
}

// Voltage of a gridded beam at channel q for the direction (s0, s1, s2) = (E, N, U), rho = sqrt(E^2 + N^2):
// bilinear interpolation in zenith angle and azimuth (east of north, periodic) of the channel's samples.
template <class G>
__device__ __forceinline__ G grid_voltage(const BeamParams &b, G s0, G s1, G rho, G s2, int q)
{
    const G kHalfPi = (G)1.5707963267948966192, kTwoPi = (G)6.283185307179586477;
    const G dth = kHalfPi / (G)(b.n_th - 1), dph = kTwoPi / (G)b.n_ph;
    const G th = atan2(rho, s2);
    G az = atan2(s0, s1);
    if (az < (G)0) az += kTwoPi;
    const G u = th / dth;
    int i = (int)floor(u);
    i = i < 0 ? 0 : (i > b.n_th - 2 ? b.n_th - 2 : i);
    const G a = u - (G)i;
    const G v = az / dph;
    const int j = (int)floor(v);
    const G c = v - (G)j;
    int j0 = j % b.n_ph;
    if (j0 < 0) j0 += b.n_ph;
    const int j1 = j0 + 1 == b.n_ph ? 0 : j0 + 1;
    const size_t base = ((size_t)q * b.n_th + i) * b.n_ph;
    G t00, t01, t10, t11;
    if (b.grid_fp64) {
        const double *T = (const double *)b.grid + base;
        t00 = (G)T[j0]; t01 = (G)T[j1]; t10 = (G)T[b.n_ph + j0]; t11 = (G)T[b.n_ph + j1];
    } else {
        const float *T = (const float *)b.grid + base;
        t00 = (G)T[j0]; t01 = (G)T[j1]; t10 = (G)T[b.n_ph + j0]; t11 = (G)T[b.n_ph + j1];
    }
    return ((G)1 - a) * (((G)1 - c) * t00 + c * t01) + a * (((G)1 - c) * t10 + c * t11);
}

// Cubic B-spline weights of the four knots around fractional offset a in [0, 1).
template <class G> __device__ __forceinline__ void bspline3(G a, G w[4])
{
    const G b = (G)1 - a, s = (G)1 / (G)6;
    w[0] = b * b * b * s;
    w[1] = ((G)3 * a * a * a - (G)6 * a * a + (G)4) * s;
    w[2] = ((G)3 * b * b * b - (G)6 * b * b + (G)4) * s;
    w[3] = a * a * a * s;
}

// The same beam by bicubic B-spline interpolation of its coefficients (zenith-angle knots mirrored
// about the end samples, azimuth periodic).
template <class G>
__device__ __forceinline__ G grid_voltage3(const BeamParams &b, G s0, G s1, G rho, G s2, int q)
{
    const G kHalfPi = (G)1.5707963267948966192, kTwoPi = (G)6.283185307179586477;
    const G dth = kHalfPi / (G)(b.n_th - 1), dph = kTwoPi / (G)b.n_ph;
    G az = atan2(s0, s1);
    if (az < (G)0) az += kTwoPi;
    const G u = atan2(rho, s2) / dth;
    int i = (int)floor(u);
    i = i < 0 ? 0 : (i > b.n_th - 2 ? b.n_th - 2 : i);
    const G v = az / dph;
    const int j = (int)floor(v);
    G wt[4], wp[4];
    bspline3<G>(u - (G)i, wt);
    bspline3<G>(v - (G)j, wp);
    int jj[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        int k = (j - 1 + c) % b.n_ph;
        jj[c] = k < 0 ? k + b.n_ph : k;
    }
    const size_t plane = (size_t)q * b.n_th * b.n_ph;
    G acc = (G)0;
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        int ii = i - 1 + r;
        ii = ii < 0 ? -ii : (ii > b.n_th - 1 ? 2 * (b.n_th - 1) - ii : ii);
        const size_t row = plane + (size_t)ii * b.n_ph;
        G sr = (G)0;
#pragma unroll
        for (int c = 0; c < 4; ++c)
            sr += wp[c] * (b.grid_fp64 ? (G)((const double *)b.grid)[row + jj[c]]
                                       : (G)((const float *)b.grid)[row + jj[c]]);
        acc += wt[r] * sr;
    }
    return acc;
}

// Beam voltage at channel q (frequency nu) for the direction (s0, s1, s2): analytic beams by
// voltage<G>, gridded beams from their samples.
template <class G>
__device__ __forceinline__ G beam_voltage(const BeamParams &b, G s0, G s1, G rho, G s2, G nu, int q)
{
    if (b.kind == 3)
        return b.grid_order == 3 ? grid_voltage3<G>(b, s0, s1, rho, s2, q) : grid_voltage<G>(b, s0, s1, rho, s2, q);
    return voltage<G>(b, rho, s2, nu);
}

// Strengths of one source in one slice (Eq. 1-2 with the slice's beams): the
// unpolarised product A_i A_j I, or the four products of J_i C J_j^dagger with
// J = A R(az) for Stokes IQUV (A_i = A_j = A for one shared beam).  Beam in the
// grid precision G.  Returns n_pol.
template <class G, class S = double>
__device__ __forceinline__ int source_strengths(const SliceGeom &g, S s0, S s1, S s2, long n,
                                                const void *flux, int flux_fp64, long n_src, int n_freq, int f,
                                                cpx<G> *c)
{
    // the beam in the grid precision (sin of the zenith angle from the direction's E, N components)
    const G e0 = (G)s0, e1 = (G)s1;
    const G rho = sqrt(e0 * e0 + e1 * e1);
    const G A = beam_voltage<G>(g.beam, e0, e1, rho, (G)s2, geom_nu<G>(g), f);
    // A_i A_j: the two antennas' voltages (one shared beam: A^2)
    const G A2 = g.two_beams ? A * beam_voltage<G>(g.beam2, e0, e1, rho, (G)s2, geom_nu<G>(g), f) : A * A;
    const void *fl = g.flux_t ? g.flux_t : flux;
    auto ld = [&](int k) -> G {
        const size_t idx = flux_index(g, k, n, n_src, n_freq, f);
        return flux_fp64 ? (G)((const double *)fl)[idx] : (G)((const float *)fl)[idx];
    };
    if (!g.polarized) {
        c[0] = cmk<G>(A2 * ld(0), (G)0);
        return 1;
    }
    const G I = ld(0), Q = ld(1), U = ld(2), V = ld(3);
    G ca = (G)1, sa = (G)0;
    if (rho > (G)0) { ca = e1 / rho; sa = e0 / rho; }
    const G c2 = ca * ca - sa * sa, s2a = (G)2 * ca * sa;
    const G Qr = Q * c2 - U * s2a, Ur = Q * s2a + U * c2;
    c[0] = cmk<G>(A2 * (I + Qr), (G)0);
    c[1] = cmk<G>(A2 * Ur, A2 * V);
    c[2] = cmk<G>(A2 * Ur, -A2 * V);
    c[3] = cmk<G>(A2 * (I - Qr), (G)0);
    return 4;
}


// ---------------------------------------------------------------- launchers
// All launchers enqueue on `st` and return the launch error (cudaSuccess if fine).

// Channel-major copy of the fluxes: out[f][n][k] = flux[k][n][f] (n_stokes k, n_src n, n_freq f), in the
// fluxes' precision.
cudaError_t launch_flux_transpose(const void *flux, int fp64, long n_src, int n_stokes, int n_freq, void *out,
                                  cudaStream_t st);

// e[3][n]: equatorial unit vectors from (ra, dec).
cudaError_t launch_radec_to_unit(const double *ra, const double *dec, long n, double *e, cudaStream_t st);

// Per-block min/max of visible ENU directions over all times: out[nblocks][6].
cudaError_t launch_source_extents(const double *e, long n, const double *R_all, int n_time,
                                  double *out, int nblocks, cudaStream_t st);

// tab[j] = 1 / Phihat(k_j), k_j = (j - n/2) * w * pi / M  (prescale table of one dim).
template <class G>
cudaError_t launch_prescale_table(G *tab, int nf1, int M, int w, double beta, const double *gl_x,
                                  const double *gl_w, int nq, cudaStream_t st);

// tw[k] = e^{2 pi i k / M}
template <class G>
cudaError_t launch_twiddles(cpx<G> *tw, int M, cudaStream_t st);

// dec[u] = prod_i (4/w^2) / Phihat(a_ui), a = (b_c - b) / b_half * w pi / (2 sigma)
// (channel-independent, Section 2.2 deconvolution), FP64.
cudaError_t launch_target_deconv(const double *bu, int n_u, int d, const double *bcen, const double *bhalf,
                                 int w, double beta, double sigma, const double *gl_x, const double *gl_w,
                                 int nq, double *dec, cudaStream_t st);

// Fused weighting (beam x flux, Eq. 1-3), rotation, horizon cut, prephase and
// spreading with global atomics onto grid [n_pol][nz][ny][nx].
template <class G>
cudaError_t launch_spread_direct(const double *e, long n_src, const void *flux, int flux_fp64, int n_freq,
                                 int f, const SliceGeom &g, cpx<G> *grid, cudaStream_t st);

// Per time: rotate, horizon cut and counting sort of the visible sources by
// top-channel tile.  sdir[3][n_src] and sidx[n_src] hold the sorted visible
// directions and source indices; offsets[nb] is the visible count.
// tc (nullable): per sorted source, the top channel's grid coordinates (s - C) qscale_top and prephase
// D_top.(s - C), computed in FP64 and stored as float pairs, and the direction in FP32:
// tc[3i] = {qx_hi, qx_lo, qy_hi, qy_lo}, tc[3i+1] = {qz_hi, qz_lo, ph_hi, ph_lo}, tc[3i+2] = {s0, s1, s2, 0}.
cudaError_t launch_time_binning(const double *e, long n_src, const TimeBin &tb, int *bin_of, int *counts,
                                int *offsets, int *cursor, double *sdir, int *sidx, float4 *tc, cudaStream_t st);

// Per slice: strengths with prephase and split grid coordinates of the sorted sources.
template <class G>
cudaError_t launch_prep(const double *sdir, const int *sidx, const int *nv_ptr, long n_src, const void *flux,
                        int flux_fp64, int n_freq, int f, const SliceGeom &g, int *cell, G *frac, cpx<G> *cs,
                        cudaStream_t st);

// Gather-spreading configuration for a grid precision, product count and z
// size: returns 0 if unsupported, else the z template size and the bin size
// (top-channel cells per bin in x and y).
int spread_gather_config(int elem_bytes, int n_pol, int nz, int w, int *nz_tmpl, int *bin_x, int *bin_y);

// Per slice: tiled spreading; writes every cell of grid [n_pol][nz][ny][nx].
template <class G>
cudaError_t launch_spread_tile(const int *offsets, const int *cell, const G *frac, const cpx<G> *cs, long n_src,
                               const SliceGeom &g, const TimeBin &tb, double r0, double r1, cpx<G> *grid,
                               cudaStream_t st);

// Scatter variant of the tiled spreading (shared-memory tile + atomics);
// same inputs and output as launch_spread_tile.
template <class G>
cudaError_t launch_spread_scatter(const int *offsets, const int *cell, const G *frac, const cpx<G> *cs, long n_src,
                                  const SliceGeom &g, const TimeBin &tb, double r0, double r1, cpx<G> *grid,
                                  cudaStream_t st);
size_t spread_scatter_smem(int elem_bytes, int n_pol, int nz);

// One FFT pass: rows of length N (input rows contiguous), prescale by pre[l],
// zero-pad to M, FFT with e^{+2 pi i l m / M}, write band outputs transposed:
// out[b][row] = P[(b - H) mod M].
template <class G>
cudaError_t launch_fft_pass(const cpx<G> *in, cpx<G> *out, long rows, const DimGeom &dg, const G *pre,
                            const cpx<G> *tw, cudaStream_t st);

// Interpolation at the unique targets, deconvolution and postphase: Vu[u][pol] (FP64).
template <class G>
cudaError_t launch_interp(const cpx<G> *band, const double *bu, int n_u, const double *dec, const SliceGeom &g,
                          cpx<double> *Vu, cudaStream_t st);

// The slice output written straight by the two-dimensional interpolation (the scatter to the baselines
// fused into it): out [n_bl][n_pol] in the grid precision; u_off[u] .. u_off[u + 1] index u_bl, the
// baselines of unique target u; u_base: the plan-wide index of the launch's first target.
struct SliceOut {
    void *out;
    const int *u_off, *u_bl;
    int u_base;
};

// Whether launch_interp_zdirect can write a slice's output itself for this geometry (two-dimensional
// grids without height terms, n_pol 1 or 4).
bool interp_fuses_scatter(const SliceGeom &g);

// Same, reading the band after the x and y passes only ([b_y][b_x][pol][l_z]),
// with the z axis summed directly (nf1_z <= 16).  so (or nullptr): write the output of the targets'
// baselines directly instead of Vu (interp_fuses_scatter must hold).
template <class G>
cudaError_t launch_interp_zdirect(const cpx<G> *band, const double *bu, int n_u, const double *dec,
                                  const SliceGeom &g, const G *prez, const cpx<G> *twz, cpx<double> *Vu,
                                  cudaStream_t st, const SliceOut *so = nullptr);

// vis slice [n_bl][n_pol] (complex128 or complex64) <- Vu[bl2u[bl]].
cudaError_t launch_scatter(const cpx<double> *Vu, const int *bl2u, int n_bl, int n_pol, void *out,
                           int out_fp64, cudaStream_t st);

// ---------------------------------------------------------------- lattice arrays (Section 2.2.1)
// Coplanar arrays whose antennas sit on a lattice x_a = x_0 + k_a1 a_1 + k_a2 a_2
// (integer k): a baseline is b = n_1 a_1 + n_2 a_2, so with x_d = kappa a_d . s
// (E, N components) a slice is V(n) = sum_s c_s exp(-i n . x_s), a type-1
// transform to the integer modes |n_d| <= H_d.
struct LatGeom {
    double a[2][2];     // lattice vectors a_d = (east, north), m
    int nf[2];          // type-1 grid points per axis (= FFT length)
    int H[2];           // largest |n_d| over the baselines
    int K;              // Chebyshev terms of the height factor (1: flat array)
};

// Per slice: strengths (no prephase), the split grid coordinates
// t_d = frac(x_d / 2 pi) nf_d of the visible sources, u = 2 up - 1 (in frac[2]), and the
// kernel values of the footprints (after frac[0..3): [n_src][2w], x then y).
template <class G>
cudaError_t launch_prep_lattice(const double *sdir, const int *sidx, const int *nv_ptr, long n_src,
                                const void *flux, int flux_fp64, int n_freq, int f, const SliceGeom &g,
                                const LatGeom &lg, int *cell, G *frac, cpx<G> *cs, cudaStream_t st);
// Spreading onto the periodic type-1 grids [K][n_pol][nf_y][nf_x] (cleared by the caller), term q
// with strengths c_s T_q(u_s): each CTA sums a block of sources into a private copy of some of the
// grids in shared memory, then adds it to the grids.
template <class G>
cudaError_t launch_spread_lattice(const int *nv_ptr, const int *cell, const G *frac, const cpx<G> *cs, long n_src,
                                  const SliceGeom &g, const LatGeom &lg, cpx<G> *grid, cudaStream_t st);
// Visibilities of the baselines from the band [b_y][b_x][q][pol] of modes m = -n
// (b_d = H_d - n_d): sum_q wq[bl][q] x band, times the deconvolution tables
// dx[n_x + H_x] dy[n_y + H_y] (wq = nullptr: K = 1 and weight 1).
// bl_list: the n_bl baselines to evaluate (one beam group), or nullptr for baselines 0..n_bl-1.
template <class G>
cudaError_t launch_gather_lattice(const cpx<G> *band, const int *bln, const int *bl_list, int n_bl, int n_pol,
                                  const LatGeom &lg, const cpx<double> *wq, const double *dx, const double *dy,
                                  void *out, int out_fp64, cudaStream_t st);
// Per-baseline height-term weights of one channel: wq[bl][q] = e^{-i beta} eps_q (-i)^q J_q(beta),
// beta = kappa b_up[bl] / 2 (FP64 series for J_q).
cudaError_t launch_lattice_wterms(const double *b_up, int n_bl, int K, double kappa, cpx<double> *wq,
                                  cudaStream_t st);
// tab[n + H] = 1 / ((w/2) Phihat(pi w n / nf)), n in [-H, H] (FP64, Gauss-Legendre quadrature)
cudaError_t launch_lattice_deconv(double *tab, int H, int nf, int w, double beta, const double *gl_x,
                                  const double *gl_w, int nq, cudaStream_t st);
// Host: lattice basis and integer indices of the antennas, or 0 (not a coplanar lattice within tol).
int lattice_detect(int n_ant, const double *enu, double tol, double basis[4], int *index);

size_t fft_pass_smem_bytes(int M, int elem_bytes);
int fft_max_M(int elem_bytes);
int fft_rows_per_cta(int M, int elem_bytes);
// Smallest even M >= target that is a product of at most 3 (4 above 4096)
// supported radices; fills radix[] and nstages.  -1 if none.
int fft_choose_length(int target, int *radix, int &nstages, int maxRadix);
// Per-stage multiply-high division constants of dg (needs M, nstages, radix).
void fft_stage_constants(DimGeom &dg);

}  // namespace fv
