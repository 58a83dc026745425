/*
 * fv.h -- C ABI of libfftvis_gb300.so, a GB300 (sm_103a) implementation of
 * the visibility hot path of fftvis (Cox et al. 2025).
 *
 * The library evaluates, for every (time, frequency) slice,
 *
 *   V^{pq}_{ij}(nu, t) = sum_n [J C_n J^dagger]_{pq} exp(-2 pi i nu b_ij . s_n(t) / c)
 *
 * (Eq. 1 with the coherency matrix of Eq. 2, under the point-source
 * approximation of Eq. 3) as one type-3 non-uniform FFT per slice (Eq. 4 with
 * x_k = -2 pi nu b_k / c, Section 2.2): beam x flux weighting, spreading with
 * the exponential-of-semicircle kernel, an oversampled FFT, deconvolution and
 * interpolation at the baselines (Fig. 1, Section 2.2 steps 1-3).  Sources are
 * rotated from equatorial coordinates to East-North-Up by the rigid rotation
 * fixed by local sidereal time and latitude (Section 2.3); one beam is shared
 * by all antennas (Section 2.2.3).
 *
 * General rules for every entry point:
 *  - Return FV_OK (0) on success or an fv_status code; no C++ exception and
 *    no CUDA error escapes.  fv_last_error() gives a message for the last
 *    failing call on a plan (valid until the next call on that plan).
 *  - Host arrays passed in are read during the call and copied; the caller
 *    keeps ownership.  Device pointers (flags *_on_device) are borrowed: they
 *    must stay valid for as long as the docs of the call say.
 *  - A plan is not thread-safe.  Use one plan per host thread.
 *  - All device work of a plan runs on one CUDA stream: the stream given in
 *    fv_opts.cuda_stream (borrowed), or one the plan creates and owns.
 *  - No CPU fallback: if no CUDA device is usable, fv_plan fails with
 *    FV_ERR_CUDA.
 */
#ifndef FV_H
#define FV_H

#ifdef __cplusplus
extern "C" {
#endif

#define FV_ABI_VERSION 5

typedef struct fv_plan_s *fv_plan_t;   /* opaque plan handle; owns its device memory */

typedef enum {
    FV_OK = 0,
    FV_ERR_ARG = 1,          /* invalid argument (NaN coordinate, size, eps range ...) */
    FV_ERR_OOM = 2,          /* device allocation failed */
    FV_ERR_CUDA = 3,         /* CUDA runtime error or no usable device */
    FV_ERR_STATE = 4,        /* call out of order (e.g. execute before set_sky) */
    FV_ERR_TIMEOUT = 5,      /* a bounded device wait ran out */
    FV_ERR_UNSUPPORTED = 6   /* valid request this build does not handle (e.g. grid too large) */
} fv_status;

typedef enum {
    FV_FP64 = 0,    /* every step in FP64; output complex128 */
    FV_MIXED = 1    /* spread, FFT and interpolation in FP32 with FP64 centring,
                       rescaling, phases and deconvolution; output complex64 */
} fv_precision;

typedef enum {
    FV_BEAM_GAUSS = 0,    /* power beam exp(-4 ln2 theta^2 / FWHM(nu)^2),
                             FWHM(nu) = beam_param[0] * beam_param[1] / nu
                             (beam_param[0] = FWHM in rad at reference frequency beam_param[1] Hz) */
    FV_BEAM_AIRY = 1,     /* voltage 2 J1(x)/x, x = pi D nu sin(theta)/c, D = beam_param[0] m */
    FV_BEAM_UNIFORM = 2,  /* A = 1 (no beam) */
    FV_BEAM_GRID = 3      /* numerical beam: samples set by fv_set_beam_grid (not accepted by fv_plan
                             or fv_set_beams, which take analytic beams only) */
} fv_beam_kind;

/* Plan options.  Analytic beams only (Section 2.4, item i); the Jones matrix of
 * the polarised path is A(theta) [[cos az, -sin az], [sin az, cos az]] with
 * the azimuth measured east of north. */
typedef struct {
    int precision;            /* fv_precision */
    double eps;               /* NUFFT tolerance (Section 2.2 and 4.2): 1e-14 <= eps <= 1e-2;
                                 FV_MIXED requires eps >= 1e-7 */
    int n_freq;               /* >= 1 */
    const double *freq_hz;    /* [n_freq] channel frequencies, > 0, copied */
    int n_time;               /* >= 1 */
    const double *lst_rad;    /* [n_time] local sidereal times, copied */
    double latitude_rad;      /* observatory latitude, |lat| <= pi/2 */
    int beam;                 /* fv_beam_kind */
    double beam_param[3];
    int polarized;            /* 0: one product (B I); 1: Stokes IQUV in, four products
                                 pq = 00, 01, 10, 11 out */
    int dims;                 /* 0: auto (3 if any baseline has b_up != 0), 2 or 3 */
    double upsampfac;         /* oversampling sigma (Section 2.2, Eq. 5); 0 = default 2.0;
                                 accepted: 1.25 <= sigma <= 3 (FV_MIXED: sigma >= 1.5, because
                                 the deconvolutions amplify FP32 rounding too much below it) */
    int kernel_width;         /* ES kernel width w in grid points; 0 = from eps
                                 (w = ceil(log10(1/eps)) + 1 at sigma = 2, Section 2.2) */
    void *cuda_stream;        /* borrowed cudaStream_t, or NULL for a plan-owned stream (so the
                                 legacy default stream is named by cudaStreamLegacy, not 0) */
    int device;               /* CUDA device ordinal; -1 = the current device */
    int n_streams;            /* slices run concurrently on this many streams, each with its own
                                 workspace (forked from and joined back to cuda_stream); 0 = 8
                                 (4 for FV_TRANSFORM_BASIS, whose times each fill the GPU) */
    int spread_method;        /* fv_spread_method; FV_SPREAD_AUTO picks the fastest that fits */
    int fft_max_radix;        /* largest FFT stage radix: 8 (fewer registers, more stages) or 16;
                                 0 = 16 */
    int transform;            /* fv_transform: which transform evaluates a slice */
    double lattice_tol_m;     /* largest distance (m) of an antenna from its lattice point, and of its
                                 height from the first antenna's, still accepted as a lattice;
                                 0 = 1e-10 m (a phase error below 2 pi nu/c x 1e-10 rad) */
    int n_basis;              /* FV_TRANSFORM_BASIS: number K of spectral basis functions,
                                 1 <= K <= min(16, n_freq), or 0 to choose K at fv_set_sky: the
                                 smallest K whose basis spectra P[(P I)(P B)] of the sources above
                                 the horizon at the first, middle and last times differ from the
                                 exact B I by at most eps in relative L2 over all sources and
                                 channels (the largest basis if none does; fv_info.basis_fit_error
                                 gives the value reached; the estimate, a difference of squared
                                 norms, resolves about 1e-8, so a smaller eps gets the largest
                                 basis); ignored by the other routes */
    int bin_size[2];          /* cells of the highest channel's grid per bin of the per-time source sort
                                 in x and y; 0 = 8 x 4; 1 <= each <= 64 */
    int heights;              /* fv_heights: how the type-3 route evaluates the up axis of a
                                 non-coplanar array (one whose baselines have b_up != 0) */
} fv_opts;

/* Up axis of a non-coplanar array on the type-3 route (Section 2.2.2 treats it
 * as the third dimension of the transform).  For arrays that are nearly flat
 * the height factor of a slice factorises:
 *   exp(-i k b_up n) = exp(-i k b_up C) exp(-i a u),  u = (n - C) / S,
 *   a = k b_up S,  k = 2 pi nu / c,
 * with n the up component of a source direction and C, S the centre and
 * half-extent of the visible sources' n (fv_info.src_centre[2],
 * src_halfwidth[2]).  Expanding exp(-i a u) = sum_q eps_q (-i)^q J_q(a) T_q(u)
 * (eps_0 = 1, else 2) and keeping the K terms whose tail bound
 * 2 sum_{q>=K} (|a|/2)^q / q! at the top channel and largest |b_up| is below
 * eps / 10 turns a slice into K two-dimensional transforms of the strengths
 * c T_q(u) that share their sources and targets; each target sums them with
 * its own weights exp(-i k b_up C) eps_q (-i)^q J_q(a).
 * FV_HEIGHTS_AUTO takes the height terms when K is at most the number of up
 * planes the three-dimensional grid of the top channel needs and the gather
 * spreading can hold K planes (n_pol K <= 32 complex sums a lane in FP32, 16
 * in FP64, K <= 16); FV_HEIGHTS_TERMS asks for them (fv_set_sky returns
 * FV_ERR_UNSUPPORTED where they cannot be used: K > 16, too many sums a lane,
 * or spread_method other than AUTO or GATHER; the call that completes the
 * plan, fv_set_sky or fv_set_array, decides); FV_HEIGHTS_GRID keeps the
 * three-dimensional grid.  fv_info.height_terms reports K (0: not taken). */
typedef enum {
    FV_HEIGHTS_AUTO = 0,
    FV_HEIGHTS_GRID = 1,
    FV_HEIGHTS_TERMS = 2
} fv_heights;

/* Transform choice (Section 2.2.1).  When the antennas' horizontal positions
 * sit on a lattice x_0 + k_1 a_1 + k_2 a_2 (integer k), every baseline is
 * n_1 a_1 + n_2 a_2 + b_up e_up and a slice is
 *   V = sum_s c_s exp(-i n . x_s) exp(-i a u_s'),  x_sd = 2 pi nu a_d . s / c,
 * a = 2 pi nu b_up / c, u_s' = up component of s.  For a flat array (b_up = 0)
 * this is the type-1 transform to the integer modes n; for small heights the
 * second factor is expanded in Chebyshev polynomials of u = 2 u_s' - 1,
 *   exp(-i a u_s') = exp(-i a/2) sum_q eps_q (-i)^q J_q(a/2) T_q(u)
 * (eps_0 = 1, else 2), truncated at the K terms whose tail bound
 * 2 sum_{q>=K} (|a|/4)^q / q! is below eps / 10, so a slice is K type-1
 * transforms with strengths c_s T_q(u_s) combined per baseline.  Each runs
 * on a periodic grid of about 2 sigma (2 max|n_d| + 1) points per axis with no
 * interpolation step.  FV_TRANSFORM_AUTO takes this route when the array is a
 * lattice, K <= 24 and K times its grid is no larger than the type-3 grid of
 * the top channel (t3 cells), and, for four products, 6 n_src K < n_src + t3
 * (the lattice spreading adds every product with global atomics into one small
 * grid, which contends for many sources); FV_TRANSFORM_TYPE3 never takes it;
 * FV_TRANSFORM_LATTICE
 * always does, and fv_set_array fails with FV_ERR_UNSUPPORTED if the array is
 * not a lattice or needs more than 24 terms.
 *
 * Spectral-basis route (Appendix A; FV_TRANSFORM_BASIS, never taken by
 * FV_TRANSFORM_AUTO).  The n_freq channels of a time share one transform per
 * function of a compact spectral basis instead of one transform per channel.
 * The basis M ([n_freq][K], K = fv_opts.n_basis) spans the polynomials of
 * degree < K in frequency (mapped to [-1, 1] over the band), with columns
 * orthonormal over the channels.  Per source, the flux coefficients
 * s_hat = M^T I (Eq. A1) and, per time, the beam coefficients
 * b_hat = M^T B(theta_n(t), nu) (Eq. A2; B = A^2, or A_i A_j with per-antenna
 * beams) give the product coefficients v_k = sum_ij s_hat_i b_hat_j d^k_ij
 * with d^k_ij = sum_q M_qi M_qj M_qk (Eqs. A3-A4).  One type-3 transform per
 * time takes the K strength vectors to the targets 2 pi nu_q b / c of every
 * channel on one grid sized for the whole band (Eq. A5), and
 * V(b, nu_q) = sum_k M_qk T_k(b, nu_q).  The result is the direct sum with each
 * source's spectrum B I replaced by P[(P I)(P B)], P = M M^T: exact when flux
 * and beam are polynomials of degree < K in frequency and for any sky at
 * K = n_freq; otherwise that truncation error adds to eps and is set by the
 * caller's choice of K (or by the plan's, n_basis = 0).  The flux coefficients
 * are recomputed by every fv_execute (a borrowed device flux may change between
 * executions); an automatic K is chosen once, at fv_set_sky.  Unpolarised plans only (fv_plan returns
 * FV_ERR_UNSUPPORTED for a polarised one).  Executed by fv_execute;
 * fv_batch_add and fv_execute_static return FV_ERR_UNSUPPORTED for such a
 * plan. */
typedef enum {
    FV_TRANSFORM_AUTO = 0,
    FV_TRANSFORM_TYPE3 = 1,
    FV_TRANSFORM_LATTICE = 2,
    FV_TRANSFORM_BASIS = 3
} fv_transform;

/* Lattice test of Section 2.2.1 on its own (host only, no device needed):
 * whether the horizontal (east, north) positions of all n_ant antennas
 * (enu_m: [n_ant][3] m) lie on one lattice within tol_m (0 = 1e-10 m).
 * Returns 1 if they do and all heights agree within tol_m, 2 if they do but
 * the heights differ, 0 if they do not.  On success basis[] = {a1_east,
 * a1_north, a2_east, a2_north} (a reduced basis: the shortest antenna
 * separation and the shortest one off its line) and index[] = [n_ant][2]
 * integer coordinates relative to antenna 0.  A collinear array gets a second
 * vector perpendicular to the first and all second coordinates 0. */
int fv_lattice_detect(int n_ant, const double *enu_m, double tol_m, double basis[4], int *index);

/* How the ES spreading step is run (all give the same result up to rounding). */
typedef enum {
    FV_SPREAD_AUTO = 0,
    FV_SPREAD_GATHER = 1,     /* per-tile, each thread sums the sources covering its cells; the tile's
                                 sorted sources are staged in shared memory by bulk asynchronous copies
                                 (FV_MIXED two-dimensional grids: persistent CTAs, a producer warp
                                 streaming chunks into a shared-memory ring, 8 x 8 blocks per warp) */
    FV_SPREAD_SCATTER = 2,    /* per-tile, warps add each source's footprint with shared atomics */
    FV_SPREAD_ATOMIC = 3,     /* one thread per source, global atomics on a cleared grid */
    FV_SPREAD_TENSOR = 4      /* an option, off by default: the gather of FV_MIXED two-dimensional grids
                                 (no height terms, n_pol 1 or 4, w <= 8) with each warp's 8 x 8 block
                                 of cells summed on the tensor cores (m16n8k8 TF32 products, three-term
                                 split for FP32 accuracy) instead of by FP32 FMAs; elsewhere it falls
                                 back to FV_SPREAD_GATHER */
} fv_spread_method;

/* Fill *o with defaults: FV_FP64, eps 1e-10, Gaussian beam 10 deg at 150 MHz,
 * unpolarised, auto dims, sigma 2, NULL stream, current device.  The caller
 * must still set freq_hz/n_freq and lst_rad/n_time. */
void fv_opts_default(fv_opts *o);

/* Create a plan on o->device.  Copies frequencies and LSTs.  Errors:
 * FV_ERR_ARG (bad option), FV_ERR_CUDA (no device), FV_ERR_OOM. */
fv_status fv_plan(const fv_opts *o, fv_plan_t *out);

/* Set the array.  enu_m: host [n_ant][3] antenna positions (East, North, Up, m).
 * pairs: host [n_bl][2] antenna index pairs (i, j), the baseline being
 * b_ij = x_i - x_j; NULL means all i < j (n_bl is then ignored and becomes
 * n_ant(n_ant-1)/2).  Identical FP64 baseline vectors share one NUFFT target
 * (the unique baseline vectors of Fig. 1, panel E), bit-exact only.
 * Errors: FV_ERR_ARG (n_ant < 1, index out of range, non-finite position). */
fv_status fv_set_array(fv_plan_t p, int n_ant, const double *enu_m, int n_bl, const int *pairs);

/* Per-antenna beams (Section 2.2.3).  Antenna a (of the array given to
 * fv_set_array) gets beam beam_of_antenna[a] of n_beams analytic beams
 * (kinds[k] a fv_beam_kind, params[3k..3k+2] its parameters as in
 * fv_opts.beam_param).  Baseline (i, j) then sees J_i C J_j^dagger with
 * J_a = A_{b(a)}(theta) R(az), and every unordered pair of beams present among
 * the baselines is one transform per slice: at most n_beams (n_beams + 1) / 2
 * transforms, each over its own baselines.  n_beams <= 0 or beam_of_antenna =
 * NULL returns to the single beam of fv_opts.  Host arrays, copied.  A new
 * fv_set_array with another antenna count also returns to the single beam.
 * Errors: FV_ERR_STATE (before fv_set_array), FV_ERR_ARG (n_beams > 16, bad
 * kind or parameter, index out of range). */
fv_status fv_set_beams(fv_plan_t p, int n_beams, const int *kinds, const double *params,
                       const int *beam_of_antenna);

/* Gridded (numerical) beam (Section 2.4, the numerically sampled beam models
 * that are interpolated to the source positions).  Beam `beam` becomes
 * FV_BEAM_GRID with the voltage samples voltage[f][i][j] (host array
 * [n_freq][n_theta][n_phi], copied) at channel f, zenith angle
 * theta_i = i (pi/2) / (n_theta - 1) (zenith to horizon) and azimuth
 * phi_j = j 2 pi / n_phi (east of north, periodic); a source's voltage is the
 * interpolation in (theta, phi) of its channel's samples, in the plan's
 * precision: order 1 bilinear, order 3 bicubic B-spline (interpolating: the
 * B-spline coefficients are solved for on the host in FP64, the zenith-angle
 * axis continued by mirror symmetry about its end samples, the azimuth axis
 * periodic), two of the orders Section 2.4 names.  The Jones matrix of the
 * polarised path is A(theta, phi) R(az) as for the analytic beams.  beam = -1
 * is the plan's beam (all antennas); beam = k >= 0 is per-antenna beam k of
 * the last fv_set_beams (a later fv_set_beams drops the per-antenna grids).
 * May be called before or after fv_set_sky; applies to later executions.
 * Errors: FV_ERR_ARG (beam out of range, n_theta < 2, n_phi < 1,
 * n_theta * n_phi > 2^22, order not 1 or 3, NULL or non-finite samples),
 * FV_ERR_OOM. */
fv_status fv_set_beam_grid(fv_plan_t p, int beam, int n_theta, int n_phi, int order, const double *voltage);

/* Set the sky: n_src point sources at (ra_rad, dec_rad), host arrays, copied.
 * flux: [n_stokes][n_src][n_freq] Jy (n_stokes = 1: I; 4: I, Q, U, V), FP64 if
 * flux_is_fp64 else FP32.  With flux_on_device = 0 it is a host array copied
 * to the device; with flux_on_device = 1 it is a device pointer borrowed until
 * the next fv_set_sky or fv_destroy (its values may be rewritten between
 * executions).  Diffuse maps enter as sources at pixel
 * centres with flux = brightness x pixel solid angle (Section 4.1).  Computes
 * the source extents over all times on the device (one synchronisation).
 * Errors: FV_ERR_ARG (n_src < 0, non-finite coordinate, n_stokes mismatch with
 * opts.polarized), FV_ERR_STATE (before fv_set_array), FV_ERR_OOM,
 * FV_ERR_UNSUPPORTED (a grid would exceed this build's size limits). */
fv_status fv_set_sky(fv_plan_t p, long n_src, const double *ra_rad, const double *dec_rad,
                     int n_stokes, const void *flux, int flux_is_fp64, int flux_on_device);

/* Compute all slices.  vis: [n_freq][n_time][n_bl][n_pol] complex values
 * (interleaved re, im), complex128 for FV_FP64 and complex64 for FV_MIXED,
 * n_pol = 4 if polarized else 1.  vis_on_device = 0: host buffer, the call
 * returns when it is filled.  vis_on_device = 1: device buffer; the call
 * returns once the work is enqueued on the plan's stream (synchronise that
 * stream before reading; a device vis must be aligned to its element size,
 * 8 or 16 bytes).  Errors: FV_ERR_STATE (no array or sky), FV_ERR_ARG (NULL
 * vis, or a device vis not aligned to its element size), FV_ERR_CUDA. */
fv_status fv_execute(fv_plan_t p, void *vis, int vis_on_device);

/* Release every device and host resource of the plan.  NULL is accepted. */
fv_status fv_destroy(fv_plan_t p);

/* Message for the last failing call on p (or on plan creation when p is NULL). */
const char *fv_last_error(fv_plan_t p);

/* Read-only plan geometry for tests, logs and the autotuner. */
typedef struct {
    int dims;             /* 2 or 3: dimensions of the type-3 transform (2 with height terms) */
    int kernel_width;     /* w */
    double beta;          /* ES shape parameter */
    double upsampfac;     /* sigma */
    int n_unique;         /* unique baseline targets */
    int n_bl;
    long n_src;
    int nf1_max[3];       /* largest spreading grid over channels, per dim (x=E, y=N, z=U) */
    int nf2_max[3];       /* largest FFT length over channels, per dim */
    double src_centre[3];     /* C: centre of the visible source directions */
    double src_halfwidth[3];  /* S: half-extent of the visible source directions */
    long long workspace_bytes;   /* device memory held by the plan */
    int transform;        /* FV_TRANSFORM_TYPE3, _LATTICE or _BASIS: the route the slices take */
    int lattice;          /* 1 if the array is a lattice (whatever the route) */
    int lattice_modes[2]; /* lattice route: modes 2 max|n_d| + 1 per axis */
    int lattice_grid[2];  /* lattice route: grid (and FFT) points per axis */
    int lattice_terms;    /* lattice route: Chebyshev terms K of the height factor (1 for a flat array) */
    double lattice_basis[4];  /* a1_east, a1_north, a2_east, a2_north (m) */
    int beam_groups;      /* transforms per slice: unordered beam pairs among the baselines (1: one beam) */
    int basis_terms;      /* spectral-basis route: K (0 on the other routes) */
    int basis_grid[3];    /* spectral-basis route: the one spreading grid of a time, per dim */
    double basis_fit_error;   /* automatic K: the estimated relative error of the basis spectra at
                                 the chosen K; -1 otherwise */
    int height_terms;     /* type-3 route of a non-coplanar array: Chebyshev terms K of the height
                             factor (fv_heights), 0 where the up axis is a grid dimension or absent;
                             dims is then 2 */
    int spread_method;    /* type-3 route: the fv_spread_method the slices use (AUTO resolved) */
} fv_info;

fv_status fv_get_info(fv_plan_t p, fv_info *info);

/* Per-kernel timing for roofline reports (no counterpart in the paper; the
 * paper times whole stages with a line profiler, Section 5).  While enabled,
 * every device launch that fv_execute (or a plain fv_batch_execute) enqueues
 * for the plan is bracketed by two CUDA events on the stream it runs on and
 * counted; fv_profile_read waits for those events, adds up the elapsed times
 * per kernel class, copies them out and resets the counters.  A batch with a
 * plan whose timing is enabled is not captured into a graph (FV_ERR_STATE).  Classes: "memset", "bin" (per-time rotation, horizon cut and
 * sort), "prep" (per-slice strengths and grid coordinates), "spread",
 * "fft_x", "fft_y", "fft_z", "interp", "scatter", "flux_t" (the channel-major
 * copy of a borrowed device flux made at each execution) (FV_PROFILE_CLASSES
 * entries; unused ones have an empty name or stay zero).
 * bytes[c] is the algorithmic HBM traffic the launches of class c imply
 * (each input read once, each output written once).  Launch counts are kept
 * even while timing is disabled. */
#define FV_PROFILE_CLASSES 12
typedef struct {
    const char *name[FV_PROFILE_CLASSES];
    double total_ms[FV_PROFILE_CLASSES];
    long long launches[FV_PROFILE_CLASSES];
    double bytes[FV_PROFILE_CLASSES];
} fv_profile_data;

fv_status fv_profile_enable(fv_plan_t p, int enable);
fv_status fv_profile_read(fv_plan_t p, fv_profile_data *out);

/* Batches: slices of many plans executed together (Section 5.4 runs (time,
 * frequency) work in parallel processes; here independent slices share the
 * GPU).  A batch owns n_lanes execution lanes (a stream and a workspace sized
 * for its largest member); plans added to a batch need no workspace of their
 * own.  Items are dealt to lanes longest first; the lanes fork from and join
 * back to the batch's stream (cuda_stream, borrowed, or NULL for an owned one).
 *  - fv_batch_add: slices t in [t_lo, t_hi), f in [f_lo, f_hi) of plan p,
 *    written into vis, a device buffer of p's full fv_execute output shape.
 *    p must stay alive and be on the batch's device until the batch is
 *    cleared or destroyed: destroying a member plan first leaves the batch
 *    (and its graph) pointing at freed memory.  A member's fv_set_sky,
 *    fv_set_array, fv_set_beams or fv_set_beam_grid is allowed: the next
 *    fv_batch_execute notices it and captures the graph again (and resizes
 *    the lanes).
 *  - fv_batch_add_range: the same slices into a buffer laid out for a
 *    window of channels from vis_f0 and vis_nt times from vis_t0: slice
 *    (t, f) goes to slice index (f - vis_f0) * vis_nt + (t - vis_t0), each
 *    slice n_bl * n_pol complex values.  The window must hold the range
 *    (vis_f0 <= f_lo, vis_t0 <= t_lo, t_hi <= vis_t0 + vis_nt, vis_nt >= 1)
 *    and vis must hold (f_hi - vis_f0) * vis_nt slices.  A request for part
 *    of a resident plan's band and times thus needs no buffer for the rest,
 *    and can be added in pieces (one time, a block of channels) that all
 *    land in the one request buffer.
 *  - fv_batch_execute: enqueues every item on the batch's stream and returns.
 *    With use_graph != 0 the first execution after a change of the item list
 *    runs once plainly, then captures the whole launch sequence into a CUDA
 *    graph; later executions replay the graph.  Graph execution needs kernel
 *    timing (fv_profile_enable) off on every member plan.
 *  - fv_batch_clear: removes all items (and the graph).
 * Errors: FV_ERR_ARG (bad range, host output, plan or output on another
 * device, output not aligned to its element size), FV_ERR_STATE, FV_ERR_OOM, FV_ERR_CUDA, FV_ERR_TIMEOUT (a bounded
 * wait of an earlier execution ran out; reported once); fv_batch_last_error
 * gives the message. */
typedef struct fv_batch_s *fv_batch_t;
/* n_lanes: 1..32, 0 = 8.  device: -1 = the current device. */
fv_status fv_batch_create(int device, void *cuda_stream, int n_lanes, fv_batch_t *out);
fv_status fv_batch_add(fv_batch_t b, fv_plan_t p, void *vis, int t_lo, int t_hi, int f_lo, int f_hi);
fv_status fv_batch_add_range(fv_batch_t b, fv_plan_t p, void *vis, int t_lo, int t_hi, int f_lo, int f_hi,
                             int vis_f0, int vis_t0, int vis_nt);
fv_status fv_batch_execute(fv_batch_t b, int use_graph);
fv_status fv_batch_clear(fv_batch_t b);
fv_status fv_batch_destroy(fv_batch_t b);
const char *fv_batch_last_error(fv_batch_t b);
/* Device memory held by the batch's lane workspaces. */
long long fv_batch_workspace_bytes(fv_batch_t b);

/* fv_execute for callers that cannot allocate device memory.  The paper has
 * no counterpart; this exists for callers such as a host framework whose own
 * allocator already owns the free HBM (a foreign cudaMalloc would fail or
 * fragment its pool), a serving loop that admits work against a fixed HBM
 * budget and must not grow while it runs, or a plug-in whose host forbids
 * device allocations outside the host's API.
 *
 * Same result as fv_execute(p, vis, 1) (same kernels, same precision), but
 * all per-slice scratch (spreading grid, FFT band buffers, source bins and
 * prepared sources, unique-target values) comes from one static device array
 * of FV_STATIC_SCRATCH_BYTES that is part of the library image; the call
 * allocates and frees nothing.  The plan (fv_plan / fv_set_array /
 * fv_set_sky) is created as usual beforehand; vis must be a device buffer of
 * the fv_execute output shape and type.
 *  - The array is committed on a device when the library's module is loaded
 *    there, which under CUDA's default lazy module loading is the first
 *    fv_execute_static call on that device; it stays until the process exits.
 *    Callers holding a fixed HBM budget make one warm-up call (a tiny plan
 *    will do) before fixing the budget.
 *  - The first call on a device (and the first after a cudaDeviceReset) looks
 *    up the array's device address (cudaGetSymbolAddress) with that device
 *    current; make that first call before any stream capture.
 *  - Every call on a device shares the one array and leaves its contents
 *    behind; the call clears what must start at zero itself.  Calls whose
 *    work overlaps on the GPU (other host threads, other plans, other
 *    streams) race on the array: serialise them.
 *  - Returns when the work is enqueued on the plan's stream.
 * Errors: FV_ERR_UNSUPPORTED if the plan needs more scratch than
 * FV_STATIC_SCRATCH_BYTES (the message gives both sizes), FV_ERR_ARG (NULL or
 * host vis, vis on another device, or vis not aligned to its element size),
 * FV_ERR_STATE, FV_ERR_CUDA,
 * FV_ERR_TIMEOUT (a bounded wait of an earlier execution ran out). */
#define FV_STATIC_SCRATCH_BYTES (64ull << 20)
fv_status fv_execute_static(fv_plan_t p, void *vis);

/* Check of the bounded waits (no counterpart in the paper).  Every wait of
 * the spreading kernels on a bulk copy gives up after about a second, records
 * the fact in the plan's device status word and returns, so that the context
 * stays usable; the plan's next execution (fv_execute, fv_execute_static or a
 * batch holding it) then returns FV_ERR_TIMEOUT once and clears the word.  This
 * call enqueues on the plan's stream one warp that waits on a barrier phase that
 * nothing completes, so its wait runs out and is recorded the same way (about a
 * second of one warp; no fault, no copy issued).  Returns FV_OK when enqueued. */
fv_status fv_selftest_wait(fv_plan_t p);

/* ABI version (FV_ABI_VERSION of the library that was loaded). */
int fv_abi_version(void);

#ifdef __cplusplus
}
#endif
#endif /* FV_H */
