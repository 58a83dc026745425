// Internal: the plan object behind fv_plan_t (shared by the runtime's
// translation units; not part of the public ABI).
#pragma once
#include "../../include/fv.h"
#include "fv_internal.cuh"

#include <string>
#include <utility>
#include <vector>

struct fv_plan_s {
    using BeamParams = fv::BeamParams;
    using SliceGeom = fv::SliceGeom;
    template <class T> using cpx = fv::cpx<T>;
    // options
    int precision = FV_FP64;
    double eps = 1e-10;
    std::vector<double> freq, lst;
    double lat = 0.0;
    BeamParams beam{};
    int polarized = 0, n_pol = 1;
    int dims_req = 0;
    // up axis of a non-coplanar array (fv_opts.heights): the array's dimension (3 if any b_up != 0), the
    // Chebyshev height terms the type-3 route takes (0: none; the transform is then d_array-dimensional)
    // and the dimension the per-target deconvolution table was computed for
    int heights_req = 0;
    int d_array = 2;
    int hK = 0;
    int dec_d = 0;
    double sigma = 2.0;
    int w = 0;
    double beta = 0.0;
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    std::string err;

    // quadrature (sine-substituted Gauss-Legendre) on the device
    int nq = 0;
    double *d_glx = nullptr, *d_glw = nullptr;

    // array (host copies kept so that fv_set_beams can regroup the baselines)
    std::vector<double> enu_h;        // [n_ant][3]
    std::vector<int> pairs_h;         // [n_bl][2]
    // per-antenna beams (Section 2.2.3): empty beams = every antenna has opts.beam
    std::vector<BeamParams> beams;
    std::vector<int> beam_of_ant;
    // gridded beams (Section 2.4): device samples of the plan's beam and of each per-antenna beam
    void *d_grid_main = nullptr;
    std::vector<void *> d_grid_beams;
    // baselines grouped by the unordered pair of their antennas' beams: group g has unique targets
    // [u0, u1) and baselines d_grp_bl[bl0, bl1) (one group covering everything without per-antenna beams)
    struct BeamGroup {
        int a = 0, b = 0;
        int u0 = 0, u1 = 0, bl0 = 0, bl1 = 0;
    };
    std::vector<BeamGroup> groups;
    int *d_grp_bl = nullptr;
    bool have_array = false;
    int n_ant = 0, n_bl = 0, n_u = 0, d = 2;
    std::vector<double> bu;          // [n_u][3]
    std::vector<int> bl2u;           // [n_bl]
    double bcen[3] = {0, 0, 0}, bhalf[3] = {0, 0, 0};
    double *d_bu = nullptr, *d_dec = nullptr;
    // per unique target, float pairs for the FP32 interpolation set-up (SliceGeom::tgt_db, tgt_bc)
    float4 *d_tgt_db = nullptr;
    float2 *d_tgt_bc = nullptr;
    int tgt_n = 0;
    std::vector<float4> h_tgt_db;
    std::vector<float2> h_tgt_bc;
    int *d_bl2u = nullptr;
    // unique target -> its baselines (CSR: d_u_off[n_u + 1] into d_u_bl[n_bl]), for the interpolation
    // that writes a slice's output itself
    int *d_u_off = nullptr, *d_u_bl = nullptr;

    // sky
    bool have_sky = false;
    long n_src = 0;
    int n_stokes = 1;
    double *d_e = nullptr;
    void *d_flux_owned = nullptr;
    // sky buffers are kept across fv_set_sky calls of the same size (allocating and freeing gigabytes of
    // fluxes each time cost more than the copies): capacities in bytes, and the small scratch of set_sky
    size_t e_bytes = 0, flux_owned_bytes = 0, flux_t_bytes = 0, radec_bytes = 0;
    double *d_radec = nullptr, *d_Rt = nullptr, *d_ext = nullptr;
    const void *flux = nullptr;
    int flux_fp64 = 0;
    // channel-major copy of the fluxes, [n_freq][n_src][n_stokes]: what the slices read (one channel's
    // Stokes values of a source adjacent).  Made at fv_set_sky from an owned copy; from a borrowed device
    // flux (which the caller may rewrite in place) at the start of every execution.
    void *d_flux_t = nullptr;
    bool flux_borrowed = false;
    double C[3] = {0, 0, 0}, S[3] = {0, 0, 0};
    bool any_visible = false;

    // geometry
    std::vector<double> Rt;          // [n_time][9]
    std::vector<SliceGeom> gf;       // per channel (R filled per time)
    std::vector<size_t> pre_off;     // [n_freq][3] element offsets into the prescale table
    std::vector<size_t> tw_off;      // [n_freq][3] element offsets into the twiddle table
    void *d_pre = nullptr, *d_tw = nullptr;
    // one workspace per execution stream (slices on different streams run concurrently)
    struct Workspace {
        void *block = nullptr;   // one allocation, carved into the pieces below
        size_t bytes = 0;
        void *grid = nullptr, *bufA = nullptr, *bufB = nullptr;
        cpx<double> *Vu = nullptr;
        int *bin_of = nullptr, *counts = nullptr, *offsets = nullptr, *cursor = nullptr, *sidx = nullptr;
        int *cell = nullptr;
        double *sdir = nullptr;
        void *frac = nullptr, *cs = nullptr;
        float4 *tc = nullptr;     // per-time coordinate records of the sorted sources (FP32 grids)
        int *tiles = nullptr;     // ring gather: ticket and work-list counts (reset by the prep kernel)
        // ring gather work list (fv_spread_ring.cu): tiles' bin rectangles, unsplit tiles, parts of split
        // tiles, per-block part counters and the parts' block sums
        int4 *ring_bins = nullptr, *ring_parts = nullptr;
        int *ring_light = nullptr, *ring_cnt = nullptr;
        float4 *ring_partial = nullptr;
        int ring_tiles = 0, ring_slots = 0;
    };
    std::vector<Workspace> ws;
    // what one execution workspace must hold for this plan (set by prepare)
    struct WsNeed {
        size_t grid = 0, bufA = 0, bufB = 0, vu = 0;   // bytes
        long n_src = 0;
        int nb = 0;
        size_t frac_per_src = 0, cs_per_src = 0;       // bytes per source
        bool tiled = false;
        bool tc = false;                               // per-time coordinate records (48 bytes per source)
        int ring_tiles = 0, ring_slots = 0, ring_np = 0; // ring gather: tiles of the largest grid, part slots, n_pol
    } need;
    int n_streams = 1;
    std::vector<cudaStream_t> sub;       // sub[0] is the plan's stream
    std::vector<cudaEvent_t> ev_join;
    cudaEvent_t ev_fork = nullptr;
    // binned spreading
    bool tiled = false;
    int spread_req = 0;         // fv_opts.spread_method
    int fft_max_radix = 16;
    int spread_method = 0;      // resolved method
    bool ring = false;          // FP32 2-D gather through the shared-memory ring (fv_spread_ring.cu)
    int bin_req[2] = {0, 0};    // fv_opts.bin_size
    int T[2] = {32, 32}, nbx = 1, nby = 1, f_top = 0;
    double qscale_top[3] = {0, 0, 0};
    int nf1_top[3] = {1, 1, 1};

    // lattice arrays (Section 2.2.1)
    int transform_req = 0;            // fv_opts.transform
    double lat_tol = 1e-10;
    bool lat_ok = false;              // the array is a lattice
    bool use_lattice = false;         // slices take the lattice route
    double lat_basis[4] = {0, 0, 0, 0};
    int lat_H[2] = {0, 0};
    int *d_bln = nullptr;             // [n_bl][2] lattice offsets n of the baselines
    fv::LatGeom lg{};
    fv::DimGeom lat_dim[2]{};         // FFT geometry of the two passes
    void *d_lat_pre = nullptr, *d_lat_tw = nullptr;   // ones (prescale) and twiddles per axis
    double *d_lat_dec = nullptr;      // 1/Psihat per axis: [2H_x+1] then [2H_y+1]
    std::vector<double> lat_bup;      // [n_bl] up component of each baseline (m)
    double *d_lat_bup = nullptr;
    cpx<double> *d_lat_wq = nullptr;  // [n_freq][n_bl][K] height-term weights (K > 1 only)

    // spectral-basis route (Appendix A): one transform per basis function and time
    int n_basis = 0;                  // K in use
    int n_basis_req = 0;              // fv_opts.n_basis (0: chosen from the sky at fv_set_sky)
    double basis_fit_err = 0.0;       // estimated relative error of the basis spectra (automatic K)
    bool use_basis = false;
    int basis_np = 1;                 // strength vectors per spreading launch (4 or 1)
    int basis_Kp = 0;                 // K rounded up to a multiple of basis_np (padded planes are zero)
    SliceGeom bg{};                   // the grid of a time, sized for the whole band
    double *d_bas_M = nullptr;        // [n_freq][K] orthonormal basis
    double *d_bas_d = nullptr;        // [K][K][K] structure constants
    double *d_bas_freq = nullptr;     // [n_freq] Hz
    double *d_bas_kappa = nullptr;    // [n_freq] 2 pi nu / c
    void *d_bas_Mg = nullptr;         // the basis and the structure constants in the grid precision
    void *d_bas_dg = nullptr;
    int4 *d_bas_tm = nullptr;         // per target (u, q): footprint origin on the FFT grid
    int *d_bas_perm = nullptr;        //   the targets of each beam group in grid order (interpolation order)
    void *d_bas_tf = nullptr;         //   offsets [4] in the grid precision
    void *d_bas_ts = nullptr;         //   deconvolution x postphase (complex, grid precision)
    double *d_bas_shat = nullptr;     // [n_src][K] flux coefficients (recomputed by every execution)

    // device status word: kernels with bounded waits or-in FV_DEVICE_TIMEOUT; copied to the pinned
    // h_status after every execution (event ev_status) and checked when that copy has landed
    int *d_status = nullptr;
    int *h_status = nullptr;
    cudaEvent_t ev_status = nullptr;
    bool status_pending = false;
    // bumped by every call that may move or replace the device buffers a captured batch graph points at
    // (fv_set_array, fv_set_sky, fv_set_beams, fv_set_beam_grid)
    unsigned long long gen = 0;

    long long ws_bytes = 0;
    std::vector<long> geo_sig;       // sizes behind the current tables and workspaces
    int nf1_max[3] = {1, 1, 1}, M_max[3] = {1, 1, 1};

    // kernel timing (fv_profile_enable)
    bool prof_on = false;
    std::vector<cudaEvent_t> ev_pool;
    std::vector<std::pair<int, int>> ev_pending;   // (class, index of the start event in the pool)
    cudaStream_t prof_stream = nullptr;
    size_t ev_next = 0;
    double prof_ms[FV_PROFILE_CLASSES] = {};
    long long prof_launches[FV_PROFILE_CLASSES] = {};
    double prof_bytes[FV_PROFILE_CLASSES] = {};
    int prof_cls = -1;

    fv_status fail(fv_status s, const std::string &m)
    {
        err = m;
        return s;
    }
    size_t elem() const { return precision == FV_FP64 ? sizeof(cpx<double>) : sizeof(cpx<float>); }
};


// Shared by the runtime's translation units.
size_t workspace_layout(const fv_plan_s::WsNeed &need, char *base, fv_plan_s::Workspace *w);
cudaError_t alloc_workspaces(const fv_plan_s::WsNeed &need, int n, std::vector<fv_plan_s::Workspace> &ws);
// Where slice (t, f) lands in an output buffer: at slice index (f - f0) * nt + (t - t0).
// The default {0, 0, 0} (nt 0 = the plan's n_time) is the plan's full [n_freq][n_time] layout.
struct OutMap {
    int f0 = 0, t0 = 0, nt = 0;
    // pinned host memory laid out like vis, or nullptr: each slice is copied there (device to host, on
    // the slice's stream) as soon as it is written, so the copies overlap the other slices' kernels
    char *host = nullptr;
};
// Slices [k_begin, k_end) (index t * n_freq + f) of plan p, on stream st with workspace wk,
// written into vis (slice_bytes per slice, placed by om).
template <class G>
fv_status run_slices(fv_plan_s *p, fv_plan_s::Workspace &wk, cudaStream_t st, char *vis, size_t slice_bytes,
                     long k_begin, long k_end, OutMap om = OutMap{});
// Spectral-basis route: times [t_begin, t_end) of plan p (all channels), on stream st with workspace wk,
// into the plan's full output layout.
template <class G>
fv_status run_basis(fv_plan_s *p, fv_plan_s::Workspace &wk, cudaStream_t st, char *vis, size_t slice_bytes,
                    int t_begin, int t_end);
// Refresh the channel-major flux copy from a borrowed device flux, on stream st (no-op otherwise).
cudaError_t refresh_flux_t(fv_plan_s *p, cudaStream_t st);
// Device status word of a plan: copy it behind an execution's work, and report (once) a bounded wait
// that ran out in an earlier execution as FV_ERR_TIMEOUT.
cudaError_t plan_post_status(fv_plan_s *p);
fv_status plan_take_status(fv_plan_s *p, bool wait);
// Orthonormal basis of the polynomials of degree < K over the channel frequencies: M[q * K + k].
bool basis_matrix(const std::vector<double> &freq, int K, std::vector<double> &M);
