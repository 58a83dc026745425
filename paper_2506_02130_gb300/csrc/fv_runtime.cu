// Host runtime and C ABI of libfftvis_gb300 (see include/fv.h).
//
// Plan-time geometry in FP64 (Section 2.2, Eq. 5 and the centring paragraph
// after it): source centre C and half-extent S from the visible directions
// over all times, target centre D and half-extent X from the baselines per
// channel, grid sizes nf1 >= 2 sigma X S / pi + w (rounded up to an even
// 2^a 3^b 5^c, at least w + 2), FFT lengths M = sigma nf1, deconvolution tables.
// Execution: per (time, channel) slice, spread -> d FFT passes -> interpolate
// -> scatter, all enqueued on the plan's stream.
#include "../../include/fv.h"
#include "fv_basis.cuh"
#include "fv_internal.cuh"
#include "fv_staged.cuh"
#include "fv_plan.cuh"

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <tuple>
#include <vector>

using namespace fv;

namespace {

thread_local std::string g_create_error;

int next235even(long n)
{
    if (n < 2) n = 2;
    if (n % 2) ++n;
    for (;; n += 2) {
        long m = n;
        while (m % 2 == 0) m /= 2;
        while (m % 3 == 0) m /= 3;
        while (m % 5 == 0) m /= 5;
        if (m == 1) return (int)n;
    }
}

// Gauss-Legendre nodes/weights on [-1, 1] by Newton iteration on P_n.
void gauss_legendre(int n, std::vector<double> &x, std::vector<double> &w)
{
    x.resize(n);
    w.resize(n);
    for (int i = 0; i < n; ++i) {
        double z = std::cos(M_PI * (i + 0.75) / (n + 0.5));
        double dp = 0.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= n; ++k) {
                double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            if (n == 1) { p1 = z; p0 = 1.0; }
            dp = n * (z * p1 - p0) / (z * z - 1.0);
            double dz = p1 / dp;
            z -= dz;
            if (std::fabs(dz) < 1e-16) break;
        }
        x[i] = z;
        w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
}

}  // namespace

#define CK(call)                                                                                        \
    do {                                                                                                \
        cudaError_t e_ = (call);                                                                        \
        if (e_ != cudaSuccess)                                                                          \
            return p->fail(e_ == cudaErrorMemoryAllocation ? FV_ERR_OOM : FV_ERR_CUDA,                  \
                           std::string(#call " failed: ") + cudaGetErrorString(e_));                  \
    } while (0)

static void dfree(void *&ptr)
{
    if (ptr) cudaFree(ptr);
    ptr = nullptr;
}
template <class T> static void dfree_t(T *&ptr)
{
    if (ptr) cudaFree(ptr);
    ptr = nullptr;
}

static const char *k_prof_names[FV_PROFILE_CLASSES] = {"memset", "bin",   "prep",    "spread",   "fft_x", "fft_y",
                                                       "fft_z",  "interp", "scatter", "flux_t", "",      ""};
enum { PC_MEMSET = 0, PC_BIN, PC_PREP, PC_SPREAD, PC_FFT_X, PC_FFT_Y, PC_FFT_Z, PC_INTERP, PC_SCATTER, PC_FLUX_T };

// harvest recorded event pairs into the per-class totals (waits for each pair's end event, so it
// holds whatever stream the launches ran on: the plan's own or a batch lane)
static cudaError_t prof_harvest(fv_plan_s *p)
{
    if (p->ev_pending.empty()) return cudaSuccess;
    cudaError_t e = cudaSuccess;
    for (auto &pr : p->ev_pending) {
        e = cudaEventSynchronize(p->ev_pool[pr.second + 1]);
        if (e != cudaSuccess) return e;
        float ms = 0.f;
        e = cudaEventElapsedTime(&ms, p->ev_pool[pr.second], p->ev_pool[pr.second + 1]);
        if (e != cudaSuccess) return e;
        p->prof_ms[pr.first] += ms;
    }
    p->ev_pending.clear();
    p->ev_next = 0;
    return cudaSuccess;
}

// bracket one launch of class cls on stream st; call prof_begin before and prof_end after it
static cudaError_t prof_begin(fv_plan_s *p, int cls, cudaStream_t st)
{
    p->prof_launches[cls] += 1;
    p->prof_cls = cls;
    p->prof_stream = st;
    if (!p->prof_on) return cudaSuccess;
    if (p->ev_next + 2 > p->ev_pool.size()) {
        // grow the pool in steps up to 8192 events, then recycle it after a harvest
        const size_t n0 = p->ev_pool.size();
        if (n0 < 8192) {
            p->ev_pool.resize(std::min<size_t>(8192, n0 + 256), nullptr);
            for (size_t i = n0; i < p->ev_pool.size(); ++i) {
                cudaError_t e = cudaEventCreate(&p->ev_pool[i]);
                if (e != cudaSuccess) return e;
            }
        } else {
            cudaError_t e = prof_harvest(p);
            if (e != cudaSuccess) return e;
        }
    }
    return cudaEventRecord(p->ev_pool[p->ev_next], st);
}

static cudaError_t prof_end(fv_plan_s *p, double bytes)
{
    p->prof_bytes[p->prof_cls] += bytes;
    if (!p->prof_on) return cudaSuccess;
    cudaError_t e = cudaEventRecord(p->ev_pool[p->ev_next + 1], p->prof_stream);
    p->ev_pending.emplace_back(p->prof_cls, (int)p->ev_next);
    p->ev_next += 2;
    return e;
}

// Carve one execution workspace for `need` out of `base` (nullptr: only size it).
size_t workspace_layout(const fv_plan_s::WsNeed &need, char *base, fv_plan_s::Workspace *w)
{
    size_t off = 0;
    auto take = [&](size_t bytes) -> void * {
        off = (off + 255) & ~(size_t)255;
        void *ptr = base ? base + off : nullptr;
        off += bytes;
        return ptr;
    };
    fv_plan_s::Workspace tmp;
    fv_plan_s::Workspace &o = w ? *w : tmp;
    o.grid = take(need.grid);
    o.bufA = take(need.bufA);
    o.bufB = take(need.bufB);
    o.Vu = (cpx<double> *)take(need.vu);
    if (need.tiled) {
        const size_t ns = (size_t)need.n_src, nb = (size_t)need.nb;
        o.bin_of = (int *)take(ns * sizeof(int));
        o.counts = (int *)take(nb * sizeof(int));
        o.offsets = (int *)take((nb + 1) * sizeof(int));
        o.cursor = (int *)take(nb * sizeof(int));
        o.sidx = (int *)take(ns * sizeof(int));
        o.cell = (int *)take(3 * ns * sizeof(int));
        o.sdir = (double *)take(3 * ns * sizeof(double));
        // 64 bytes of slack: the band spreader's bulk copies round their ends up to 16 bytes
        o.frac = take(ns * need.frac_per_src + 64);
        o.cs = take(ns * need.cs_per_src + 64);
        o.tc = need.tc ? (float4 *)take(ns * 3 * sizeof(float4)) : nullptr;
        o.tiles = (int *)take(4 * sizeof(int));
        if (need.ring_tiles > 0) {
            const size_t nt = (size_t)need.ring_tiles, sl = (size_t)need.ring_slots;
            o.ring_tiles = need.ring_tiles;
            o.ring_slots = need.ring_slots;
            o.ring_bins = (int4 *)take(nt * sizeof(int4));
            o.ring_light = (int *)take(nt * sizeof(int));
            o.ring_cnt = (int *)take(nt * kRingBlocks * sizeof(int));
            o.ring_parts = (int4 *)take(sl * sizeof(int4));
            o.ring_partial = (float4 *)take(sl * kRingBlocks * need.ring_np * 32 * sizeof(float4));
        }
    }
    return off;
}

// Allocate n workspaces for `need` (one cudaMalloc each).
cudaError_t alloc_workspaces(const fv_plan_s::WsNeed &need, int n, std::vector<fv_plan_s::Workspace> &ws)
{
    const size_t bytes = workspace_layout(need, nullptr, nullptr);
    ws.assign(n, fv_plan_s::Workspace{});
    for (auto &w : ws) {
        cudaError_t e = cudaMalloc(&w.block, std::max<size_t>(bytes, 256));
        if (e != cudaSuccess) return e;
        w.bytes = bytes;
        workspace_layout(need, (char *)w.block, &w);
    }
    return cudaSuccess;
}

static void free_workspaces(std::vector<fv_plan_s::Workspace> &ws)
{
    for (auto &w : ws)
        if (w.block) cudaFree(w.block);
    ws.clear();
}

// Device samples of the per-antenna gridded beams (dropped with the beams they belong to).
static void drop_beam_grids(fv_plan_s *p)
{
    for (auto &d : p->d_grid_beams) dfree(d);
    p->d_grid_beams.clear();
}

static void free_geometry(fv_plan_s *p)
{
    dfree(p->d_pre);
    dfree(p->d_tw);
    dfree(p->d_lat_pre);
    dfree(p->d_lat_tw);
    dfree_t(p->d_lat_dec);
    dfree_t(p->d_lat_bup);
    dfree_t(p->d_lat_wq);
    dfree_t(p->d_bas_M);
    dfree_t(p->d_bas_d);
    dfree_t(p->d_bas_freq);
    dfree_t(p->d_bas_kappa);
    dfree(p->d_bas_Mg);
    dfree(p->d_bas_dg);
    dfree_t(p->d_bas_tm);
    dfree_t(p->d_bas_perm);
    dfree(p->d_bas_tf);
    dfree(p->d_bas_ts);
    dfree_t(p->d_bas_shat);
    free_workspaces(p->ws);
}

// Top channel, spreading method and bin geometry (needs the per-channel geometry).
static void resolve_spread(fv_plan_s *p, int gs, int w)
{
    const int nf = (int)p->freq.size();
    p->f_top = 0;
    for (int f = 1; f < nf; ++f)
        if (p->freq[f] > p->freq[p->f_top]) p->f_top = f;
    for (int i = 0; i < 3; ++i) {
        p->qscale_top[i] = p->gf[p->f_top].dim[i].qscale;
        p->nf1_top[i] = p->gf[p->f_top].dim[i].nf1;
    }
    const int nzm = p->d == 3 ? p->nf1_max[2] : (p->hK > 0 ? p->hK : 1);
    int nz_t = 0, bx = 8, by = 4;
    const bool gather_ok = spread_gather_config(gs, p->n_pol, nzm, w, &nz_t, &bx, &by) != 0;
    const bool scatter_ok = spread_scatter_smem(gs, p->n_pol, nzm) <= FV_SPREAD_SMEM_MAX && w <= 32;
    // FP64 tiles of 16 height planes hold 16 double-complex accumulators per lane: measured slower than
    // the other methods for the per-channel slices, so auto takes them only where nothing else exists
    const bool gather_auto = gather_ok && !(gs == 8 && nz_t > 8);
    // the ring gather (and its tensor-core form): FP32 two-dimensional grids without height terms
    const bool ring_ok = gather_ok && gs == 4 && p->d == 2 && p->hK == 0 && (p->n_pol == 1 || p->n_pol == 4) &&
                         w <= kRingWmax && p->precision == FV_MIXED;
    int m = p->spread_req;
    if (m == FV_SPREAD_TENSOR && !ring_ok) m = FV_SPREAD_GATHER;
    if (m == FV_SPREAD_AUTO)
        m = ring_ok || gather_auto ? FV_SPREAD_GATHER : (scatter_ok ? FV_SPREAD_SCATTER : FV_SPREAD_ATOMIC);
    if (p->hK > 0) m = FV_SPREAD_GATHER;    // the height terms are spread by the gather kernel only (checked)
    if (m == FV_SPREAD_GATHER && !gather_ok) m = FV_SPREAD_ATOMIC;
    if (m == FV_SPREAD_SCATTER && !scatter_ok) m = FV_SPREAD_ATOMIC;
    p->spread_method = m;
    p->ring = ring_ok && (m == FV_SPREAD_GATHER || m == FV_SPREAD_TENSOR);
    p->tiled = m != FV_SPREAD_ATOMIC;
    // bins of the per-time sort: the plan's size, else 8 x 4 cells of the top channel's grid
    p->T[0] = p->bin_req[0] > 0 ? p->bin_req[0] : 8;
    p->T[1] = p->bin_req[1] > 0 ? p->bin_req[1] : 4;
    p->nbx = (p->nf1_top[0] + p->T[0] - 1) / p->T[0];
    p->nby = (p->nf1_top[1] + p->T[1] - 1) / p->T[1];
}

// The lattice route (Section 2.2.1): grid and FFT geometry per axis, prescale (ones), twiddles and
// deconvolution tables, and the workspace it needs; taken if the array is a lattice and, in auto
// mode, its grid is no larger than the type-3 grid of the top channel.
static fv_status prepare_lattice(fv_plan_s *p)
{
    p->use_lattice = false;
    if (!p->lat_ok || p->transform_req == FV_TRANSFORM_TYPE3 || p->dims_req == 3) return FV_OK;
    const int w = p->w;
    LatGeom lg{};
    DimGeom dg[2]{};
    long cells = 1;
    for (int k = 0; k < 2; ++k) {
        lg.a[k][0] = p->lat_basis[2 * k];
        lg.a[k][1] = p->lat_basis[2 * k + 1];
        lg.H[k] = p->lat_H[k];
        const int B = 2 * lg.H[k] + 1;
        const int target = std::max((int)std::ceil(p->sigma * B - 1e-9), 2 * w);
        DimGeom &d = dg[k];
        d.M = fft_choose_length(target + (target & 1), d.radix, d.nstages, p->fft_max_radix);
        if (d.M < 0 || d.M > fft_max_M((int)(p->precision == FV_FP64 ? sizeof(double) : sizeof(float))))
            return p->fail(FV_ERR_UNSUPPORTED, "lattice grid too large");
        d.nf1 = d.M;
        d.H = lg.H[k];
        d.B = B;
        fft_stage_constants(d);
        lg.nf[k] = d.M;
        cells *= d.M;
    }
    // Chebyshev terms of the height factor: the tail 2 sum_{q>=K} (beta/2)^q / q! below eps / 10
    double bup_max = 0.0;
    for (double v : p->lat_bup) bup_max = std::max(bup_max, std::fabs(v));
    const double beta = 0.5 * 2.0 * M_PI * p->freq[p->f_top] / FV_C_LIGHT * bup_max;
    int K = 1;
    if (bup_max > 0.0) {
        const double h = 0.5 * beta;
        for (K = 1; K <= 64; ++K) {
            double term = 1.0, tail = 0.0;
            for (int q = 1; q <= K; ++q) term *= h / q;          // (beta/2)^K / K!
            for (int q = K; q < K + 60; ++q) {
                tail += term;
                term *= h / (q + 1);
            }
            if (2.0 * tail <= 0.1 * p->eps) break;
        }
    }
    lg.K = K;
    const DimGeom *top = p->gf[p->f_top].dim;
    const long t3 = (long)top[0].nf1 * top[1].nf1 * top[2].nf1;     // up planes or height terms included
    if (K > 24) {
        if (p->transform_req == FV_TRANSFORM_LATTICE)
            return p->fail(FV_ERR_UNSUPPORTED, "the lattice route would need " + std::to_string(K) +
                                                   " height terms (at most 24)");
        return FV_OK;
    }
    if (p->transform_req == FV_TRANSFORM_AUTO && cells * K > t3) return FV_OK;
    // four products: the lattice spreading adds every product of every source with global atomics into one
    // small grid, which contends; measured per slice on the 350-antenna workload (886k sources, K = 1) the
    // lattice route took 0.52 ms against the type-3 route's 0.20 ms (about 6 N K units against N + t3 for
    // the type-3 spreading and FFT passes), so auto keeps polarised plans on the type-3 route unless
    // 6 N K < N + t3
    if (p->transform_req == FV_TRANSFORM_AUTO && p->n_pol == 4 &&
        6.0 * (double)p->n_src * K >= (double)p->n_src + (double)t3)
        return FV_OK;
    p->use_lattice = true;
    p->lg = lg;
    p->lat_dim[0] = dg[0];
    p->lat_dim[1] = dg[1];
    const size_t es = p->elem();
    const size_t gs = p->precision == FV_FP64 ? sizeof(double) : sizeof(float);
    dfree(p->d_lat_pre);
    dfree(p->d_lat_tw);
    dfree_t(p->d_lat_dec);
    const size_t npre = (size_t)lg.nf[0] + lg.nf[1];
    CK(cudaMalloc(&p->d_lat_pre, npre * gs));
    CK(cudaMalloc(&p->d_lat_tw, npre * es));
    CK(cudaMalloc(&p->d_lat_dec, (size_t)(2 * lg.H[0] + 1 + 2 * lg.H[1] + 1) * sizeof(double)));
    if (p->precision == FV_FP64) {
        std::vector<double> ones(npre, 1.0);
        CK(cudaMemcpyAsync(p->d_lat_pre, ones.data(), npre * gs, cudaMemcpyHostToDevice, p->stream));
        CK(launch_twiddles<double>((cpx<double> *)p->d_lat_tw, lg.nf[0], p->stream));
        CK(launch_twiddles<double>((cpx<double> *)p->d_lat_tw + lg.nf[0], lg.nf[1], p->stream));
    } else {
        std::vector<float> ones(npre, 1.0f);
        CK(cudaMemcpyAsync(p->d_lat_pre, ones.data(), npre * gs, cudaMemcpyHostToDevice, p->stream));
        CK(launch_twiddles<float>((cpx<float> *)p->d_lat_tw, lg.nf[0], p->stream));
        CK(launch_twiddles<float>((cpx<float> *)p->d_lat_tw + lg.nf[0], lg.nf[1], p->stream));
    }
    CK(launch_lattice_deconv(p->d_lat_dec, lg.H[0], lg.nf[0], w, p->beta, p->d_glx, p->d_glw, p->nq, p->stream));
    CK(launch_lattice_deconv(p->d_lat_dec + 2 * lg.H[0] + 1, lg.H[1], lg.nf[1], w, p->beta, p->d_glx, p->d_glw,
                             p->nq, p->stream));
    dfree_t(p->d_lat_bup);
    dfree_t(p->d_lat_wq);
    if (K > 1 && p->n_bl > 0) {
        const int nf = (int)p->freq.size();
        CK(cudaMalloc(&p->d_lat_bup, (size_t)p->n_bl * sizeof(double)));
        CK(cudaMemcpyAsync(p->d_lat_bup, p->lat_bup.data(), (size_t)p->n_bl * sizeof(double), cudaMemcpyHostToDevice,
                           p->stream));
        CK(cudaMalloc(&p->d_lat_wq, (size_t)nf * p->n_bl * K * sizeof(cpx<double>)));
        for (int f = 0; f < nf; ++f)
            CK(launch_lattice_wterms(p->d_lat_bup, p->n_bl, K, 2.0 * M_PI * p->freq[f] / FV_C_LIGHT,
                                     p->d_lat_wq + (size_t)f * p->n_bl * K, p->stream));
    }
    // workspace of one lattice slice: grid, the two bands, one-bin time binning, prepared sources
    fv_plan_s::WsNeed nd;
    const int np = p->n_pol;
    nd.grid = (size_t)K * np * lg.nf[0] * lg.nf[1] * es;
    nd.bufA = (size_t)(2 * lg.H[0] + 1) * K * np * lg.nf[1] * es;
    nd.bufB = (size_t)(2 * lg.H[1] + 1) * (2 * lg.H[0] + 1) * K * np * es;
    nd.vu = sizeof(cpx<double>);
    nd.tiled = true;
    nd.n_src = std::max<long>(p->n_src, 1);
    nd.nb = 1;
    nd.frac_per_src = (3 + 2 * (size_t)w) * gs;     // fx, fy, u and the 2w kernel values
    nd.cs_per_src = (size_t)np * es;
    free_workspaces(p->ws);
    p->need = nd;
    p->ws_bytes = (long long)(npre * (gs + es) + p->n_streams * workspace_layout(nd, nullptr, nullptr) +
                              (K > 1 ? p->freq.size() * (size_t)p->n_bl * K * sizeof(cpx<double>) : 0));
    return FV_OK;
}

// Per-channel geometry, tables and workspace; needs the array and the sky.
// Grid and FFT geometry of one dimension of a transform whose targets have half-extent X and whose
// sources have half-extent S (Eq. 5: nf1 >= 2 sigma X S / pi + w); D and C are left to the caller.
static fv_status dim_geometry(fv_plan_s *p, double X, double S, DimGeom &dg)
{
    const int w = p->w;
    const int maxM = fft_max_M((int)(p->precision == FV_FP64 ? sizeof(double) : sizeof(float)));
    if (!(X > 0.0)) X = S > 0.0 ? 1.0 / S : 1.0;
    double need = 2.0 * p->sigma * X * S / M_PI + w;
    long nf1 = (long)std::ceil(need);
    if (nf1 < w + 1) nf1 = w + 1;     // Eq. 5 is the requirement; no 2w floor is needed
    if (nf1 > (1L << 20)) return p->fail(FV_ERR_UNSUPPORTED, "spreading grid too large");
    dg.nf1 = next235even(nf1);
    dg.M = fft_choose_length((int)std::ceil(p->sigma * dg.nf1 - 1e-9), dg.radix, dg.nstages, p->fft_max_radix);
    if (dg.M < 0 || dg.M > maxM)
        return p->fail(FV_ERR_UNSUPPORTED, "FFT length " + std::to_string(dg.M) + " exceeds " +
                                               std::to_string(maxM) + " for one-CTA FFT passes");
    dg.H = (int)std::ceil(dg.M / (2.0 * p->sigma) + 0.5 * w) + 1;
    dg.B = 2 * dg.H + 1;
    dg.qscale = p->sigma * X / M_PI;
    dg.pscale = dg.M / (2.0 * p->sigma * X);
    fft_stage_constants(dg);
    return FV_OK;
}

static fv_status prepare_basis(fv_plan_s *p);

// Height terms (fv_heights) of a non-coplanar array on the type-3 route: K from the tail bound of the
// Jacobi-Anger expansion at the top channel and the largest |b_up|, taken where the options allow it and
// the gather spreading can hold K planes (automatic: where K is at most the up planes of the top channel's
// three-dimensional grid).  Sets p->d (2 with height terms, else the array's) and p->hK, and recomputes
// the per-target deconvolution table when its dimension changes.
static fv_status choose_heights(fv_plan_s *p)
{
    p->d = p->d_array;
    p->hK = 0;
    const bool asked = p->heights_req == FV_HEIGHTS_TERMS;
    const bool may = asked || (p->heights_req == FV_HEIGHTS_AUTO && p->dims_req == 0);
    if (p->d_array == 3 && may && !p->use_basis) {
        const int nf = (int)p->freq.size();
        int f_top = 0;
        for (int f = 1; f < nf; ++f)
            if (p->freq[f] > p->freq[f_top]) f_top = f;
        double bup_max = 0.0;
        for (int u = 0; u < p->n_u; ++u) bup_max = std::max(bup_max, std::fabs(p->bu[3 * (size_t)u + 2]));
        const double kappa_top = 2.0 * M_PI * p->freq[f_top] / FV_C_LIGHT;
        const double a = kappa_top * bup_max * p->S[2];
        // smallest K with 2 sum_{q>=K} (a/2)^q / q! <= eps / 10 (|J_q(a)| <= (a/2)^q / q!)
        int K = 1;
        if (a > 0.0) {
            const double h = 0.5 * a;
            for (K = 1; K <= 64; ++K) {
                double term = 1.0, tail = 0.0;
                for (int q = 1; q <= K; ++q) term *= h / q;
                for (int q = K; q < K + 60; ++q) {
                    tail += term;
                    term *= h / (q + 1);
                }
                if (2.0 * tail <= 0.1 * p->eps) break;
            }
        }
        // FP32 grids of one product: an even K (one more term where the bound gives an odd one), so that the
        // interpolation reads the terms of a footprint cell in pairs
        if (p->precision == FV_MIXED && p->n_pol == 1 && K > 1 && (K & 1)) ++K;
        const int gs = p->precision == FV_FP64 ? (int)sizeof(double) : (int)sizeof(float);
        int nzt = 0, bx = 0, by = 0;
        const bool fits = K <= 16 && spread_gather_config(gs, p->n_pol, K, p->w, &nzt, &bx, &by) != 0 &&
                          (p->spread_req == FV_SPREAD_AUTO || p->spread_req == FV_SPREAD_GATHER);
        if (asked && !fits)
            return p->fail(FV_ERR_UNSUPPORTED, "heights = FV_HEIGHTS_TERMS: " + std::to_string(K) +
                                                   " height terms do not fit the gather spreading (at most 16, "
                                                   "n_pol K complex sums a lane within its budget, spread_method "
                                                   "AUTO or GATHER)");
        bool take = fits;
        if (take && !asked) {
            // the up planes the three-dimensional grid of the top channel would take
            DimGeom dz{};
            const fv_status ds = dim_geometry(p, kappa_top * p->bhalf[2], p->S[2], dz);
            take = ds != FV_OK || K <= dz.nf1;
            p->err.clear();
        }
        if (take) {
            p->d = 2;
            p->hK = K;
        }
    }
    if (p->dec_d != p->d && p->n_u > 0) {
        CK(launch_target_deconv(p->d_bu, p->n_u, p->d, p->bcen, p->bhalf, p->w, p->beta, p->sigma, p->d_glx,
                                p->d_glw, p->nq, p->d_dec, p->stream));
        p->dec_d = p->d;
    }
    return FV_OK;
}

static fv_status prepare(fv_plan_s *p)
{
    const fv_status hs = choose_heights(p);
    if (hs != FV_OK) return hs;
    if (p->use_basis) return prepare_basis(p);
    const int nf = (int)p->freq.size();
    const int w = p->w;
    p->gf.assign(nf, SliceGeom{});
    p->pre_off.assign((size_t)nf * 3, 0);
    p->tw_off.assign((size_t)nf * 3, 0);
    size_t pre_total = 0, tw_total = 0;
    for (int i = 0; i < 3; ++i) { p->nf1_max[i] = 1; p->M_max[i] = 1; }
    size_t grid_e = 0, bufA_e = 0, bufB_e = 0;
    for (int f = 0; f < nf; ++f) {
        SliceGeom &g = p->gf[f];
        g.nu = p->freq[f];
        g.kappa = 2.0 * M_PI * g.nu / FV_C_LIGHT;
        g.d = p->d;
        g.w = w;
        g.beta = p->beta;
        g.nu_f = (float)g.nu;
        g.beta_f = (float)g.beta;
        g.n_pol = p->n_pol;
        g.polarized = p->polarized;
        g.n_stokes = p->n_stokes;
        g.beam = p->beam;
        g.K = p->hK;
        g.hc = p->C[2];
        g.hs = p->S[2] > 0.0 ? p->S[2] : 1.0;
        g.hc_f = (float)g.hc;
        g.hs_inv_f = (float)(1.0 / g.hs);
        for (int i = 0; i < 3; ++i) {
            DimGeom &dg = g.dim[i];
            if (i >= p->d) {
                // no grid dimension: one plane, or the K planes of the height terms
                dg.nf1 = i == 2 && p->hK > 0 ? p->hK : 1;
                dg.M = 1; dg.B = 1; dg.H = 0; dg.qscale = 0; dg.pscale = 0; dg.D = 0; dg.C = 0;
                dg.nstages = 0;
                continue;
            }
            const fv_status ds = dim_geometry(p, g.kappa * p->bhalf[i], p->S[i], dg);
            if (ds != FV_OK) return ds;
            dg.D = -g.kappa * p->bcen[i];
            dg.C = p->C[i];
            p->nf1_max[i] = std::max(p->nf1_max[i], dg.nf1);
            p->M_max[i] = std::max(p->M_max[i], dg.M);
            p->pre_off[(size_t)f * 3 + i] = pre_total;
            pre_total += dg.nf1;
            p->tw_off[(size_t)f * 3 + i] = tw_total;
            tw_total += dg.M;
        }
        for (int i = 0; i < 2; ++i) {
            const double a = g.kappa * g.dim[i].pscale;
            g.a_hi[i] = (float)a;
            g.a_lo[i] = (float)(a - (double)g.a_hi[i]);
        }
        g.kap_hi = (float)g.kappa;
        g.kap_lo = (float)(g.kappa - (double)g.kap_hi);
        // buffer sizes (complex elements) for this channel
        const DimGeom *D = g.dim;
        size_t grid_c = (size_t)p->n_pol * D[0].nf1 * D[1].nf1 * D[2].nf1;
        size_t pass1 = (size_t)D[0].B * p->n_pol * D[2].nf1 * D[1].nf1;
        size_t pass2 = (size_t)D[1].B * D[0].B * p->n_pol * D[2].nf1;
        size_t pass3 = p->d == 3 ? (size_t)D[2].B * D[1].B * D[0].B * p->n_pol : 0;
        grid_e = std::max(grid_e, grid_c);
        bufA_e = std::max(bufA_e, std::max(pass1, pass3));
        bufB_e = std::max(bufB_e, pass2);
    }
    const size_t es = p->elem();
    const size_t gs = p->precision == FV_FP64 ? sizeof(double) : sizeof(float);
    // a new sky with the same grid sizes (the usual case: same array, same channels) keeps the
    // tables and workspaces of the previous one
    std::vector<long> sig = {(long)p->n_src, (long)p->n_pol, (long)p->n_streams, (long)p->spread_req, (long)p->d,
                             (long)p->hK,
                             (long)grid_e, (long)bufA_e, (long)bufB_e, (long)p->lat_ok, (long)p->lat_H[0],
                             (long)p->lat_H[1], (long)p->n_u, (long)p->n_bl};
    for (int k = 0; k < 4; ++k) {
        long long bits;
        std::memcpy(&bits, &p->lat_basis[k], sizeof(bits));
        sig.push_back((long)bits);
    }
    for (int f = 0; f < nf; ++f)
        for (int i = 0; i < 3; ++i) {
            sig.push_back(p->gf[f].dim[i].nf1);
            sig.push_back(p->gf[f].dim[i].M);
        }
    // per-target float pairs of the FP32 interpolation set-up (they depend on the sky's centre C)
    if (p->n_u > 0) {
        if (p->tgt_n != p->n_u) {
            dfree_t(p->d_tgt_db);
            dfree_t(p->d_tgt_bc);
            CK(cudaMalloc(&p->d_tgt_db, (size_t)p->n_u * sizeof(float4)));
            CK(cudaMalloc(&p->d_tgt_bc, (size_t)p->n_u * sizeof(float2)));
            p->tgt_n = p->n_u;
        }
        p->h_tgt_db.resize(p->n_u);
        p->h_tgt_bc.resize(p->n_u);
        auto pair = [](double v, float &hi, float &lo) {
            hi = (float)v;
            lo = (float)(v - (double)hi);
        };
        for (int u = 0; u < p->n_u; ++u) {
            const double *b = &p->bu[3 * (size_t)u];
            float4 &t = p->h_tgt_db[u];
            pair(b[0] - p->bcen[0], t.x, t.y);
            pair(b[1] - p->bcen[1], t.z, t.w);
            double bc = 0.0;
            for (int i = 0; i < p->d; ++i) bc += b[i] * p->C[i];
            pair(bc, p->h_tgt_bc[u].x, p->h_tgt_bc[u].y);
        }
        CK(cudaMemcpyAsync(p->d_tgt_db, p->h_tgt_db.data(), (size_t)p->n_u * sizeof(float4), cudaMemcpyHostToDevice,
                           p->stream));
        CK(cudaMemcpyAsync(p->d_tgt_bc, p->h_tgt_bc.data(), (size_t)p->n_u * sizeof(float2), cudaMemcpyHostToDevice,
                           p->stream));
    }
    const bool reuse = p->d_pre != nullptr && sig == p->geo_sig;
    if (!reuse) free_geometry(p);
    p->geo_sig.clear();
    if (reuse) {
        resolve_spread(p, (int)gs, w);
        p->geo_sig = sig;
        return FV_OK;        // the lattice route's tables and decision depend on the array only: kept
    }
    CK(cudaMalloc(&p->d_pre, std::max<size_t>(pre_total, 1) * gs));
    CK(cudaMalloc(&p->d_tw, std::max<size_t>(tw_total, 1) * es));
    p->need.grid = std::max<size_t>(grid_e, 1) * es;
    p->need.bufA = std::max<size_t>(bufA_e, 1) * es;
    p->need.bufB = std::max<size_t>(bufB_e, 1) * es;
    p->need.vu = std::max<size_t>((size_t)p->n_u * p->n_pol, 1) * sizeof(cpx<double>);
    for (int f = 0; f < nf; ++f) {
        for (int i = 0; i < p->d; ++i) {
            const DimGeom &dg = p->gf[f].dim[i];
            if (p->precision == FV_FP64) {
                CK(launch_prescale_table<double>((double *)p->d_pre + p->pre_off[(size_t)f * 3 + i], dg.nf1, dg.M, w,
                                                 p->beta, p->d_glx, p->d_glw, p->nq, p->stream));
                CK(launch_twiddles<double>((cpx<double> *)p->d_tw + p->tw_off[(size_t)f * 3 + i], dg.M, p->stream));
            } else {
                CK(launch_prescale_table<float>((float *)p->d_pre + p->pre_off[(size_t)f * 3 + i], dg.nf1, dg.M, w,
                                                p->beta, p->d_glx, p->d_glw, p->nq, p->stream));
                CK(launch_twiddles<float>((cpx<float> *)p->d_tw + p->tw_off[(size_t)f * 3 + i], dg.M, p->stream));
            }
        }
    }
    resolve_spread(p, (int)gs, w);
    p->need.tiled = p->tiled;
    p->need.n_src = std::max<long>(p->n_src, 1);
    p->need.nb = p->nbx * p->nby;
    // the gather spreading reads staged records: 16 (FP32) or 32 (FP64) bytes per source where the split
    // coordinates take 12 or 24, and strengths padded to 16 bytes
    const bool staged = p->spread_method == FV_SPREAD_GATHER || p->spread_method == FV_SPREAD_TENSOR;
    p->need.frac_per_src = p->ring ? sizeof(RingRec) : (staged ? 4 * gs : 3 * gs);
    // ring gather: a work list over the tiles of the largest grid, and slots for the parts of split tiles
    // (a tile's candidates come to at most 4 n_src, split tiles have more than kRingPart candidates each,
    // so there are at most 8 n_src / kRingPart parts; beyond kRingSlotsMax tiles run whole)
    p->need.ring_tiles = p->ring ? ring_tiles(p->nf1_max[0], p->nf1_max[1]) : 0;
    p->need.ring_slots = p->ring ? (int)std::min<long>(kRingSlotsMax, 8 * std::max<long>(p->n_src, 1) / kRingPart + 1) : 0;
    p->need.ring_np = p->ring ? p->n_pol : 0;
    p->need.cs_per_src = staged ? (size_t)staged_cs_stride((int)gs, p->n_pol) * es : (size_t)p->n_pol * es;
    // FP32 grids take each slice's coordinates and prephase from per-time records (no FP64 per slice)
    p->need.tc = p->precision == FV_MIXED && p->tiled;
    const size_t bin_bytes = p->tiled ? workspace_layout(p->need, nullptr, nullptr) -
                                            (p->need.grid + p->need.bufA + p->need.bufB + p->need.vu)
                                      : 0;
    p->ws_bytes = (long long)(pre_total * gs + tw_total * es +
                              p->n_streams * ((grid_e + bufA_e + bufB_e) * es +
                                              (size_t)p->n_u * p->n_pol * sizeof(cpx<double>) + bin_bytes));
    fv_status ls = prepare_lattice(p);
    if (ls != FV_OK) return ls;
    CK(cudaStreamSynchronize(p->stream));
    p->geo_sig = sig;
    return FV_OK;
}

// Slice geometry of channel f at time t for beam group gr: the group's two beams (Section 2.2.3;
// one shared beam: opts.beam and A^2).

static SliceGeom slice_geom_for(const fv_plan_s *p, int f, int t, const fv_plan_s::BeamGroup &gr)
{
    SliceGeom g = p->gf[f];
    g.flux_t = p->d_flux_t;
    const double r = p->gf[f].kappa / p->gf[p->f_top].kappa;
    g.rsc_hi = (float)r;
    g.rsc_lo = (float)(r - (double)g.rsc_hi);
    std::memcpy(g.R, &p->Rt[(size_t)t * 9], 9 * sizeof(double));
    if (!p->beams.empty()) {
        g.beam = p->beams[gr.a];
        g.beam2 = p->beams[gr.b];
        g.two_beams = gr.a != gr.b;
    } else {
        g.two_beams = 0;
    }
    beam_float_constant(g.beam);
    beam_float_constant(g.beam2);
    return g;
}

// Slices of a lattice array (Section 2.2.1): one-bin time binning (rotation and horizon cut), then per
// slice strengths and periodic grid coordinates, spreading, the two FFT passes without padding, and the
// per-baseline mode lookup with deconvolution.
template <class G>
static fv_status run_slices_lattice(fv_plan_s *p, fv_plan_s::Workspace &wk, cudaStream_t st, char *vis,
                                    size_t slice_bytes, long k_begin, long k_end, OutMap om)
{
    const int nf = (int)p->freq.size(), nt = (int)p->lst.size();
    const LatGeom &lg = p->lg;
    const int np = p->n_pol;
    const double es = sizeof(cpx<G>);
    cpx<G> *grid = (cpx<G> *)wk.grid, *A = (cpx<G> *)wk.bufA, *Bb = (cpx<G> *)wk.bufB;
    const G *pre = (const G *)p->d_lat_pre;
    const cpx<G> *tw = (const cpx<G> *)p->d_lat_tw;
    const size_t gel = (size_t)lg.K * np * lg.nf[0] * lg.nf[1];
    const int Bx = 2 * lg.H[0] + 1, By = 2 * lg.H[1] + 1;
    const double nvis = 0.5 * p->n_src;
    int t_binned = -1;
    for (long k = k_begin; k < k_end; ++k) {
        const int t = (int)(k / nf), f = (int)(k % nf);
        if (t != t_binned) {
            TimeBin tb{};
            std::memcpy(tb.R, &p->Rt[(size_t)t * 9], 9 * sizeof(double));
            for (int i = 0; i < 3; ++i) tb.nf1_top[i] = 1;
            tb.T[0] = tb.T[1] = 1;
            tb.nbx = tb.nby = 1;
            CK(prof_begin(p, PC_BIN, st));
            CK(launch_time_binning(p->d_e, p->n_src, tb, wk.bin_of, wk.counts, wk.offsets, wk.cursor, wk.sdir,
                                   wk.sidx, nullptr, st));
            CK(prof_end(p, (double)p->n_src * 80.0));
            t_binned = t;
        }
        // one set of transforms per beam group (Section 2.2.3), evaluated at the group's baselines
        const bool single = p->groups.size() == 1;
        for (const auto &gr : p->groups) {
            const int nbl = gr.bl1 - gr.bl0;
            if (nbl <= 0) continue;
            SliceGeom g = slice_geom_for(p, f, t, gr);
            G *frac = (G *)wk.frac;
            cpx<G> *cs = (cpx<G> *)wk.cs;
            CK(prof_begin(p, PC_PREP, st));
            CK(launch_prep_lattice<G>(wk.sdir, wk.sidx, wk.offsets + 1, p->n_src, p->flux, p->flux_fp64, nf, f, g, lg,
                                      wk.cell, frac, cs, st));
            CK(prof_end(p, nvis * (24.0 + 4.0 + p->n_stokes * (p->flux_fp64 ? 8.0 : 4.0) + 8.0 + 2.0 * sizeof(G) +
                                   np * es)));
            CK(prof_begin(p, PC_MEMSET, st));
            CK(cudaMemsetAsync(grid, 0, gel * sizeof(cpx<G>), st));
            CK(prof_end(p, gel * es));
            CK(prof_begin(p, PC_SPREAD, st));
            CK(launch_spread_lattice<G>(wk.offsets + 1, wk.cell, frac, cs, p->n_src, g, lg, grid, st));
            CK(prof_end(p, nvis * (8.0 + 3.0 * sizeof(G) + np * es) + gel * es));
            const long r1 = (long)lg.K * np * lg.nf[1];
            CK(prof_begin(p, PC_FFT_X, st));
            CK(launch_fft_pass<G>(grid, A, r1, p->lat_dim[0], nullptr, tw, st));      // no prescale (ones)
            CK(prof_end(p, (double)r1 * (lg.nf[0] + Bx) * es));
            const long r2 = (long)Bx * lg.K * np;
            CK(prof_begin(p, PC_FFT_Y, st));
            CK(launch_fft_pass<G>(A, Bb, r2, p->lat_dim[1], nullptr, tw + lg.nf[0], st));
            CK(prof_end(p, (double)r2 * (lg.nf[1] + By) * es));
            const int ntm = om.nt > 0 ? om.nt : nt;
            char *out = vis + ((size_t)(f - om.f0) * ntm + (t - om.t0)) * slice_bytes;
            CK(prof_begin(p, PC_INTERP, st));
            const cpx<double> *wq = p->d_lat_wq ? p->d_lat_wq + (size_t)f * p->n_bl * lg.K : nullptr;
            CK(launch_gather_lattice<G>(Bb, p->d_bln, single ? nullptr : p->d_grp_bl + gr.bl0, nbl, np, lg, wq,
                                        p->d_lat_dec, p->d_lat_dec + Bx, out,
                                        p->precision == FV_FP64, st));
            CK(prof_end(p, (double)nbl * (8.0 + lg.K * (np * es + (wq ? 16.0 : 0.0))) + (double)slice_bytes));
        }
        if (om.host) {
            const int ntm = om.nt > 0 ? om.nt : nt;
            const size_t off = ((size_t)(f - om.f0) * ntm + (t - om.t0)) * slice_bytes;
            CK(cudaMemcpyAsync(om.host + off, vis + off, slice_bytes, cudaMemcpyDeviceToHost, st));
        }
    }
    return FV_OK;
}

template <class G>
fv_status run_slices(fv_plan_s *p, fv_plan_s::Workspace &wk, cudaStream_t st, char *vis, size_t slice_bytes,
                     long k_begin, long k_end, OutMap om)
{
    if (p->use_basis)
        return p->fail(FV_ERR_UNSUPPORTED, "the spectral-basis route runs whole times: use fv_execute");
    if (p->use_lattice) return run_slices_lattice<G>(p, wk, st, vis, slice_bytes, k_begin, k_end, om);
    const int nf = (int)p->freq.size(), nt = (int)p->lst.size();
    cpx<G> *grid = (cpx<G> *)wk.grid;
    cpx<G> *A = (cpx<G> *)wk.bufA, *Bb = (cpx<G> *)wk.bufB;
    const double es = sizeof(cpx<G>);
    const double src_bytes = (double)p->n_src * (3 * sizeof(double) + (double)p->n_stokes * (p->flux_fp64 ? 8 : 4));
    // prep and spread touch the visible sources only; about half the sky is up at any time
    const double nvis = 0.5 * p->n_src;
    const double prep_bytes = nvis * (24.0 + 4.0 + p->n_stokes * (p->flux_fp64 ? 8.0 : 4.0) + 12.0 +
                                      3.0 * sizeof(G) + p->n_pol * es);
    // staged records: one 16- or 32-byte record (80 bytes with the ring gather's kernel values) plus the
    // (padded) strengths per source, read once
    const bool ring = p->ring && sizeof(G) == 4 && p->need.tc;
    const double rec_bytes = ring ? (double)sizeof(RingRec) : (double)sizeof(SrcRec<G>);
    const double cs_staged = staged_cs_stride((int)sizeof(G), p->n_pol) * es;
    const double prep_bytes_staged = nvis * ((p->need.tc && sizeof(G) == 4 ? 48.0 : 24.0) + 4.0 +
                                             p->n_stokes * (p->flux_fp64 ? 8.0 : 4.0) + rec_bytes + cs_staged);
    const int nb = p->nbx * p->nby;
    const G *pre = (const G *)p->d_pre;
    const cpx<G> *tw = (const cpx<G> *)p->d_tw;
    int t_binned = -1;
    TimeBin tb{};
    for (long k = k_begin; k < k_end; ++k) {
        const int t = (int)(k / nf), f = (int)(k % nf);
        if (p->tiled && t != t_binned) {
            std::memcpy(tb.R, &p->Rt[(size_t)t * 9], 9 * sizeof(double));
            for (int i = 0; i < 3; ++i) {
                tb.C[i] = p->C[i];
                tb.qscale_top[i] = p->qscale_top[i];
                tb.nf1_top[i] = p->nf1_top[i];
            }
            tb.T[0] = p->T[0];
            tb.T[1] = p->T[1];
            tb.nbx = p->nbx;
            tb.nby = p->nby;
            tb.d = p->d;
            for (int i = 0; i < 3; ++i) tb.D_top[i] = p->gf[p->f_top].dim[i].D;
            CK(prof_begin(p, PC_BIN, st));
            CK(launch_time_binning(p->d_e, p->n_src, tb, wk.bin_of, wk.counts, wk.offsets, wk.cursor, wk.sdir,
                                   wk.sidx, sizeof(G) == 4 ? wk.tc : nullptr, st));
            CK(prof_end(p, (double)p->n_src * 80.0 + nb * 12.0 + (wk.tc ? p->n_src * 0.5 * 48.0 : 0.0)));
            t_binned = t;
        }
        const int ntm = om.nt > 0 ? om.nt : nt;
        char *out = vis + ((size_t)(f - om.f0) * ntm + (t - om.t0)) * slice_bytes;
        // two-dimensional grids: the interpolation writes the baselines' output itself (no scatter)
        const bool fused = p->d == 2 && p->hK == 0 && p->d_u_off && interp_fuses_scatter(p->gf[f]);
        // one transform per beam group: strengths with the group's two beams, targets [u0, u1)
        for (const auto &gr : p->groups) {
            if (gr.u1 <= gr.u0) continue;
            SliceGeom g = slice_geom_for(p, f, t, gr);
            g.tgt_db = p->d_tgt_db && p->tgt_n == p->n_u ? p->d_tgt_db + gr.u0 : nullptr;
            g.tgt_bc = g.tgt_db ? p->d_tgt_bc + gr.u0 : nullptr;
            const int nug = gr.u1 - gr.u0;
            const double *bug = p->d_bu + 3 * (size_t)gr.u0, *decg = p->d_dec + gr.u0;
            cpx<double> *Vug = wk.Vu + (size_t)gr.u0 * p->n_pol;
            const DimGeom *D = g.dim;
            const size_t gel = (size_t)p->n_pol * D[0].nf1 * D[1].nf1 * D[2].nf1;
            if (p->tiled) {
                G *frac = (G *)wk.frac;
                cpx<G> *cs = (cpx<G> *)wk.cs;
                // the gather spreading reads staged records (bulk-copied per chunk)
                const bool staged = p->spread_method == FV_SPREAD_GATHER || p->spread_method == FV_SPREAD_TENSOR;
                SrcRec<G> *rec = (SrcRec<G> *)wk.frac;
                CK(prof_begin(p, PC_PREP, st));
                if (sizeof(G) == 4 && wk.tc)
                    CK(launch_prep_tc(wk.tc, wk.sidx, wk.offsets + nb, p->n_src, p->flux, p->flux_fp64, nf, f, g,
                                      wk.cell, (float *)frac, (cpx<float> *)cs,
                                      staged && !ring ? (SrcRec<float> *)rec : nullptr,
                                      ring ? (RingRec *)wk.frac : nullptr, ring ? wk.tiles : nullptr, st));
                else if (staged)
                    CK(launch_prep_staged<G>(wk.sdir, wk.sidx, wk.offsets + nb, p->n_src, p->flux, p->flux_fp64, nf,
                                             f, g, rec, cs, st));
                else
                    CK(launch_prep<G>(wk.sdir, wk.sidx, wk.offsets + nb, p->n_src, p->flux, p->flux_fp64, nf, f, g,
                                      wk.cell, frac, cs, st));
                CK(prof_end(p, staged ? prep_bytes_staged : prep_bytes));
                const double r0 = D[0].qscale / p->qscale_top[0], r1 = D[1].qscale / p->qscale_top[1];
                g.pre_x = pre + p->pre_off[(size_t)f * 3];         // applied as the tile is stored
                g.pre_y = pre + p->pre_off[(size_t)f * 3 + 1];
                CK(prof_begin(p, PC_SPREAD, st));
                if (ring)
                    CK(launch_spread_ring(wk.offsets, (const RingRec *)wk.frac, (const cpx<float> *)cs, g, tb, r0, r1,
                                          RingWork{wk.tiles, wk.ring_bins, wk.ring_light, wk.ring_parts, wk.ring_cnt,
                                                   wk.ring_partial, wk.ring_tiles, wk.ring_slots},
                                          p->d_status, (cpx<float> *)grid, p->spread_method == FV_SPREAD_TENSOR, st));
                else if (p->spread_method == FV_SPREAD_GATHER || p->spread_method == FV_SPREAD_TENSOR)
                    CK(launch_spread_gather_rec<G>(wk.offsets, rec, cs, g, tb, r0, r1, p->d_status, grid, st));
                else if (p->spread_method == FV_SPREAD_SCATTER)
                    CK(launch_spread_scatter<G>(wk.offsets, wk.cell, frac, cs, p->n_src, g, tb, r0, r1, grid, st));
                else
                    CK(launch_spread_tile<G>(wk.offsets, wk.cell, frac, cs, p->n_src, g, tb, r0, r1, grid, st));
                // algorithmic bytes of the spreading step, whatever the staging: the visible sources' fluxes
                // read once and the grid written once (the records and strengths it reads are the prep's
                // output, counted there)
                CK(prof_end(p, nvis * p->n_stokes * (p->flux_fp64 ? 8.0 : 4.0) + gel * es));
            } else {
                CK(prof_begin(p, PC_MEMSET, st));
                CK(cudaMemsetAsync(grid, 0, gel * sizeof(cpx<G>), st));
                CK(prof_end(p, gel * es));
                CK(prof_begin(p, PC_SPREAD, st));
                CK(launch_spread_direct<G>(p->d_e, p->n_src, p->flux, p->flux_fp64, nf, f, g, grid, st));
                CK(prof_end(p, src_bytes + gel * es));
            }
            const size_t o0 = (size_t)f * 3;
            // the tiled spreading kernels stored the grid with its x and y prescale already applied
            const G *pre_x = p->tiled ? nullptr : pre + p->pre_off[o0];
            const G *pre_y = p->tiled ? nullptr : pre + p->pre_off[o0 + 1];
            // pass 1 along x: rows (pol, z, y)
            const long r1 = (long)p->n_pol * D[2].nf1 * D[1].nf1;
            CK(prof_begin(p, PC_FFT_X, st));
            CK(launch_fft_pass<G>(grid, A, r1, D[0], pre_x, tw + p->tw_off[o0], st));
            CK(prof_end(p, (double)r1 * (D[0].nf1 + D[0].B) * es));
            // pass 2 along y: rows (bx, pol, z)
            const long r2 = (long)D[0].B * p->n_pol * D[2].nf1;
            CK(prof_begin(p, PC_FFT_Y, st));
            CK(launch_fft_pass<G>(A, Bb, r2, D[1], pre_y, tw + p->tw_off[o0 + 1], st));
            CK(prof_end(p, (double)r2 * (D[1].nf1 + D[1].B) * es));
            if (p->d == 2 || D[2].nf1 <= FV_ZDIRECT_MAX) {
                // z (if any) summed directly inside the interpolation: no z pass
                const double wd = (double)p->w * p->w * D[2].nf1;
                CK(prof_begin(p, PC_INTERP, st));
                const SliceOut so{out, p->d_u_off, p->d_u_bl, gr.u0};
                CK(launch_interp_zdirect<G>(Bb, bug, nug, decg, g, pre + p->pre_off[o0 + 2],
                                            tw + p->tw_off[o0 + 2], Vug, st, fused ? &so : nullptr));
                // with the scatter fused in, the baselines' output is written here
                const double nbl_g = gr.bl1 - gr.bl0;
                CK(prof_end(p, (double)nug * (wd * p->n_pol * es + 4 * sizeof(double) + p->n_pol * 16.0) +
                                   (fused ? nbl_g * 4.0 + (double)slice_bytes * nbl_g / std::max(p->n_bl, 1) : 0.0)));
            } else {
                // pass 3 along z: rows (by, bx, pol)
                const long r3 = (long)D[1].B * D[0].B * p->n_pol;
                CK(prof_begin(p, PC_FFT_Z, st));
                CK(launch_fft_pass<G>(Bb, A, r3, D[2], pre + p->pre_off[o0 + 2], tw + p->tw_off[o0 + 2], st));
                CK(prof_end(p, (double)r3 * (D[2].nf1 + D[2].B) * es));
                const double wd = std::pow((double)p->w, p->d);
                CK(prof_begin(p, PC_INTERP, st));
                CK(launch_interp<G>(A, bug, nug, decg, g, Vug, st));
                CK(prof_end(p, (double)nug * (wd * p->n_pol * es + 4 * sizeof(double) + p->n_pol * 16.0)));
            }
        }
        if (!fused) {
            CK(prof_begin(p, PC_SCATTER, st));
            CK(launch_scatter(wk.Vu, p->d_bl2u, p->n_bl, p->n_pol, out, p->precision == FV_FP64, st));
            CK(prof_end(p, (double)p->n_bl * (4 + p->n_pol * 16.0) + (double)slice_bytes));
        }
        if (om.host) CK(cudaMemcpyAsync(om.host + (out - vis), out, slice_bytes, cudaMemcpyDeviceToHost, st));
    }
    return FV_OK;
}

template fv_status run_slices<float>(fv_plan_s *, fv_plan_s::Workspace &, cudaStream_t, char *, size_t, long, long,
                                     OutMap);
template fv_status run_slices<double>(fv_plan_s *, fv_plan_s::Workspace &, cudaStream_t, char *, size_t, long, long,
                                      OutMap);

// The spectral-basis route (Appendix A): the basis and its structure constants, one grid per time
// sized for the targets of every channel (Eq. A5), its FFT tables, the deconvolution of every
// (baseline, channel) target and the workspace.
// Automatic K (n_basis = 0): the smallest K whose spectra P[(P I)(P B)] of the sources above the
// horizon at the first, middle and last times differ from the exact B I by at most eps in relative L2
// over all sources and channels (measured on the device with the largest basis the channels allow);
// K = that largest basis if none does.
static fv_status choose_basis_terms(fv_plan_s *p)
{
    const int nf = (int)p->freq.size(), nt = (int)p->lst.size();
    std::vector<double> M;
    int Kmax = std::min(kBasisMax, nf);
    while (Kmax > 1 && !basis_matrix(p->freq, Kmax, M)) --Kmax;
    if (Kmax <= 1 || p->n_src == 0 || !p->any_visible) {
        p->n_basis = 1;
        p->basis_fit_err = 0.0;
        return FV_OK;
    }
    std::vector<double> dK((size_t)Kmax * Kmax * Kmax, 0.0);
    for (int i = 0; i < Kmax; ++i)
        for (int j = 0; j < Kmax; ++j)
            for (int k = 0; k < Kmax; ++k) {
                double acc = 0.0;
                for (int q = 0; q < nf; ++q)
                    acc += M[(size_t)q * Kmax + i] * M[(size_t)q * Kmax + j] * M[(size_t)q * Kmax + k];
                dK[((size_t)i * Kmax + j) * Kmax + k] = acc;
            }
    std::vector<int> ts = {0, nt / 2, nt - 1};
    ts.erase(std::unique(ts.begin(), ts.end()), ts.end());
    std::vector<double> R;
    for (int t : ts) R.insert(R.end(), p->Rt.begin() + (size_t)t * 9, p->Rt.begin() + (size_t)t * 9 + 9);
    BeamParams b1 = p->beam, b2 = p->beam;
    int two = 0;
    if (!p->beams.empty() && !p->groups.empty()) {
        b1 = p->beams[p->groups[0].a];
        b2 = p->beams[p->groups[0].b];
        two = p->groups[0].a != p->groups[0].b;
    }
    double *d = nullptr;
    const size_t nM = M.size(), nD = dK.size(), nR = R.size();
    CK(cudaMalloc(&d, (nM + nD + nR + nf + Kmax + 1) * sizeof(double)));
    double *dM = d, *dD = dM + nM, *dR = dD + nD, *dF = dR + nR, *dErr = dF + nf;
    cudaError_t e = cudaMemcpyAsync(dM, M.data(), nM * sizeof(double), cudaMemcpyHostToDevice, p->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dD, dK.data(), nD * sizeof(double), cudaMemcpyHostToDevice, p->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dR, R.data(), nR * sizeof(double), cudaMemcpyHostToDevice, p->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dF, p->freq.data(), nf * sizeof(double), cudaMemcpyHostToDevice, p->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(dErr, 0, (Kmax + 1) * sizeof(double), p->stream);
    if (e == cudaSuccess)
        e = launch_basis_fit(p->d_e, p->n_src, dR, (int)ts.size(), p->flux, p->flux_fp64, nf, dF, dM, dD, Kmax, b1,
                             b2, two, dErr, p->stream);
    std::vector<double> err(Kmax + 1, 0.0);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(err.data(), dErr, (Kmax + 1) * sizeof(double), cudaMemcpyDeviceToHost, p->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(p->stream);
    cudaFree(d);
    if (e != cudaSuccess) return p->fail(FV_ERR_CUDA, cudaGetErrorString(e));
    const double total = err[Kmax];
    int K = Kmax;
    double r = 0.0;
    for (int k = 1; k <= Kmax; ++k) {
        const double rk = total > 0.0 ? std::sqrt(std::max(err[k - 1], 0.0) / total) : 0.0;
        r = rk;
        if (rk <= p->eps) {
            K = k;
            break;
        }
    }
    p->n_basis = K;
    p->basis_fit_err = r;
    return FV_OK;
}

static fv_status prepare_basis(fv_plan_s *p)
{
    if (p->n_basis_req == 0) {
        const fv_status ks = choose_basis_terms(p);
        if (ks != FV_OK) return ks;
    }
    const int nf = (int)p->freq.size(), K = p->n_basis, w = p->w;
    const size_t gs = p->precision == FV_FP64 ? sizeof(double) : sizeof(float);
    const size_t es = p->elem();
    std::vector<double> M;
    if (!basis_matrix(p->freq, K, M))
        return p->fail(FV_ERR_ARG, "n_basis exceeds the number of distinct channel frequencies");
    std::vector<double> dK((size_t)K * K * K, 0.0);
    for (int i = 0; i < K; ++i)
        for (int j = 0; j < K; ++j)
            for (int k = 0; k < K; ++k) {
                double acc = 0.0;
                for (int q = 0; q < nf; ++q) acc += M[(size_t)q * K + i] * M[(size_t)q * K + j] * M[(size_t)q * K + k];
                dK[((size_t)i * K + j) * K + k] = acc;
            }
    std::vector<double> kappa(nf);
    double kmin = INFINITY, kmax = 0.0;
    for (int q = 0; q < nf; ++q) {
        kappa[q] = 2.0 * M_PI * p->freq[q] / FV_C_LIGHT;
        kmin = std::min(kmin, kappa[q]);
        kmax = std::max(kmax, kappa[q]);
    }
    // targets x = -kappa b: over the baselines' box and kappa in [kmin, kmax] the extremes sit at the
    // box corners and the two ends of the band
    SliceGeom g{};
    g.nu = 0.0;
    g.kappa = 1.0;
    g.d = p->d;
    g.w = w;
    g.beta = p->beta;
    g.beta_f = (float)p->beta;
    g.polarized = 0;
    g.n_stokes = 1;
    g.beam = p->beam;
    double Xc[3] = {1, 1, 1};
    for (int i = 0; i < 3; ++i) {
        DimGeom &dg = g.dim[i];
        if (i >= p->d) {
            dg.nf1 = 1; dg.M = 1; dg.B = 1; dg.H = 0; dg.qscale = 0; dg.pscale = 0; dg.D = 0; dg.C = 0;
            dg.nstages = 0;
            continue;
        }
        const double blo = p->bcen[i] - p->bhalf[i], bhi = p->bcen[i] + p->bhalf[i];
        const double xlo = std::min(-kmin * bhi, -kmax * bhi), xhi = std::max(-kmin * blo, -kmax * blo);
        const fv_status ds = dim_geometry(p, 0.5 * (xhi - xlo), p->S[i], dg);
        if (ds != FV_OK) return ds;
        dg.D = 0.5 * (xhi + xlo);
        dg.C = p->C[i];
        Xc[i] = dg.qscale * M_PI / p->sigma;      // the half-extent the geometry used (after the X = 0 fix-up)
    }
    const int nz = p->d == 3 ? g.dim[2].nf1 : 1;
    if (nz > FV_ZDIRECT_MAX)
        return p->fail(FV_ERR_UNSUPPORTED, "spectral-basis route: the grid's height axis is too long for the direct sum");
    int nzt = 0, bx = 0, by = 0;
    const int np = spread_gather_config((int)gs, 4, nz, w, &nzt, &bx, &by) ? 4
                   : (spread_gather_config((int)gs, 1, nz, w, &nzt, &bx, &by) ? 1 : 0);
    if (np == 0 || K * nz > 256)
        return p->fail(FV_ERR_UNSUPPORTED, "spectral-basis route: no spreading kernel for this grid depth");
    g.n_pol = np;
    p->basis_np = np;
    p->basis_Kp = (K + np - 1) / np * np;
    p->bg = g;
    // bins over the one grid of a time
    p->spread_method = FV_SPREAD_GATHER;
    p->tiled = true;
    p->f_top = 0;
    p->T[0] = 8;
    p->T[1] = 4;
    for (int i = 0; i < 3; ++i) {
        p->nf1_top[i] = g.dim[i].nf1;
        p->qscale_top[i] = g.dim[i].qscale;
        p->nf1_max[i] = g.dim[i].nf1;
        p->M_max[i] = g.dim[i].M;
    }
    p->nbx = (p->nf1_top[0] + p->T[0] - 1) / p->T[0];
    p->nby = (p->nf1_top[1] + p->T[1] - 1) / p->T[1];
    // tables
    free_geometry(p);
    p->geo_sig.clear();
    p->pre_off.assign(3, 0);
    p->tw_off.assign(3, 0);
    size_t pre_total = 0, tw_total = 0;
    for (int i = 0; i < p->d; ++i) {
        p->pre_off[i] = pre_total;
        pre_total += g.dim[i].nf1;
        p->tw_off[i] = tw_total;
        tw_total += g.dim[i].M;
    }
    CK(cudaMalloc(&p->d_pre, std::max<size_t>(pre_total, 1) * gs));
    CK(cudaMalloc(&p->d_tw, std::max<size_t>(tw_total, 1) * es));
    for (int i = 0; i < p->d; ++i) {
        const DimGeom &dg = g.dim[i];
        if (p->precision == FV_FP64) {
            CK(launch_prescale_table<double>((double *)p->d_pre + p->pre_off[i], dg.nf1, dg.M, w, p->beta, p->d_glx,
                                             p->d_glw, p->nq, p->stream));
            CK(launch_twiddles<double>((cpx<double> *)p->d_tw + p->tw_off[i], dg.M, p->stream));
        } else {
            CK(launch_prescale_table<float>((float *)p->d_pre + p->pre_off[i], dg.nf1, dg.M, w, p->beta, p->d_glx,
                                            p->d_glw, p->nq, p->stream));
            CK(launch_twiddles<float>((cpx<float> *)p->d_tw + p->tw_off[i], dg.M, p->stream));
        }
    }
    CK(cudaMalloc(&p->d_bas_M, M.size() * sizeof(double)));
    CK(cudaMalloc(&p->d_bas_d, dK.size() * sizeof(double)));
    CK(cudaMalloc(&p->d_bas_freq, nf * sizeof(double)));
    CK(cudaMalloc(&p->d_bas_kappa, nf * sizeof(double)));
    CK(cudaMalloc(&p->d_bas_shat, (size_t)std::max<long>(p->n_src, 1) * K * sizeof(double)));
    CK(cudaMemcpyAsync(p->d_bas_M, M.data(), M.size() * sizeof(double), cudaMemcpyHostToDevice, p->stream));
    CK(cudaMemcpyAsync(p->d_bas_d, dK.data(), dK.size() * sizeof(double), cudaMemcpyHostToDevice, p->stream));
    CK(cudaMemcpyAsync(p->d_bas_freq, p->freq.data(), nf * sizeof(double), cudaMemcpyHostToDevice, p->stream));
    CK(cudaMemcpyAsync(p->d_bas_kappa, kappa.data(), nf * sizeof(double), cudaMemcpyHostToDevice, p->stream));
    // the basis and structure constants in the grid precision, and the constants of every target (u, q)
    std::vector<float> Mf(M.begin(), M.end()), dKf(dK.begin(), dK.end());
    CK(cudaMalloc(&p->d_bas_Mg, M.size() * gs));
    CK(cudaMalloc(&p->d_bas_dg, dK.size() * gs));
    const size_t nt_all = (size_t)p->n_u * nf;
    CK(cudaMalloc(&p->d_bas_tm, std::max<size_t>(nt_all, 1) * sizeof(int4)));
    CK(cudaMalloc(&p->d_bas_tf, std::max<size_t>(nt_all, 1) * 4 * gs));
    CK(cudaMalloc(&p->d_bas_ts, std::max<size_t>(nt_all, 1) * es));
    if (p->precision == FV_FP64) {
        CK(cudaMemcpyAsync(p->d_bas_Mg, M.data(), M.size() * gs, cudaMemcpyHostToDevice, p->stream));
        CK(cudaMemcpyAsync(p->d_bas_dg, dK.data(), dK.size() * gs, cudaMemcpyHostToDevice, p->stream));
        CK(launch_basis_targets<double>(p->d_bu, p->n_u, p->d_bas_kappa, nf, g, Xc, p->sigma, p->d_glx, p->d_glw,
                                        p->nq, p->d_bas_tm, (double *)p->d_bas_tf, (cpx<double> *)p->d_bas_ts,
                                        p->stream));
    } else {
        CK(cudaMemcpyAsync(p->d_bas_Mg, Mf.data(), M.size() * gs, cudaMemcpyHostToDevice, p->stream));
        CK(cudaMemcpyAsync(p->d_bas_dg, dKf.data(), dK.size() * gs, cudaMemcpyHostToDevice, p->stream));
        CK(launch_basis_targets<float>(p->d_bu, p->n_u, p->d_bas_kappa, nf, g, Xc, p->sigma, p->d_glx, p->d_glw,
                                       p->nq, p->d_bas_tm, (float *)p->d_bas_tf, (cpx<float> *)p->d_bas_ts,
                                       p->stream));
    }
    // the interpolation takes each beam group's targets sorted by footprint row, then column, so that the
    // warps of a CTA, and consecutive CTAs, read overlapping parts of the band
    std::vector<int4> tmh(std::max<size_t>(nt_all, 1));
    CK(cudaMemcpyAsync(tmh.data(), p->d_bas_tm, nt_all * sizeof(int4), cudaMemcpyDeviceToHost, p->stream));
    CK(cudaStreamSynchronize(p->stream));
    std::vector<int> perm(std::max<size_t>(nt_all, 1));
    for (size_t t = 0; t < nt_all; ++t) perm[t] = (int)t;
    for (const auto &gr : p->groups) {
        auto lo = perm.begin() + (size_t)gr.u0 * nf, hi = perm.begin() + (size_t)gr.u1 * nf;
        std::sort(lo, hi, [&](int a, int b) {
            const int4 &A = tmh[a], &B = tmh[b];
            return A.y != B.y ? A.y < B.y : (A.x != B.x ? A.x < B.x : a < b);
        });
    }
    CK(cudaMalloc(&p->d_bas_perm, perm.size() * sizeof(int)));
    CK(cudaMemcpyAsync(p->d_bas_perm, perm.data(), perm.size() * sizeof(int), cudaMemcpyHostToDevice, p->stream));
    CK(cudaStreamSynchronize(p->stream));
    // workspace of one execution stream
    const DimGeom *D = g.dim;
    p->need = fv_plan_s::WsNeed{};
    p->need.grid = (size_t)p->basis_Kp * D[0].nf1 * D[1].nf1 * D[2].nf1 * es;
    p->need.bufA = (size_t)D[0].B * K * D[2].nf1 * D[1].nf1 * es;
    p->need.bufB = (size_t)D[1].B * D[0].B * K * D[2].nf1 * es;
    p->need.vu = std::max<size_t>(nt_all, 1) * sizeof(cpx<double>);
    p->need.tiled = true;
    p->need.n_src = std::max<long>(p->n_src, 1);
    p->need.nb = p->nbx * p->nby;
    p->need.frac_per_src = 3 * gs;
    p->need.cs_per_src = (size_t)p->basis_Kp * es;
    p->ws_bytes = (long long)(pre_total * gs + tw_total * es + (M.size() + dK.size() + 2 * nf) * (8 + gs) +
                              nt_all * (sizeof(int4) + sizeof(int) + 4 * gs + es) +
                              (size_t)p->need.n_src * K * 8 +
                              p->n_streams * workspace_layout(p->need, nullptr, nullptr));
    return FV_OK;
}

template <class G>
fv_status run_basis(fv_plan_s *p, fv_plan_s::Workspace &wk, cudaStream_t st, char *vis, size_t slice_bytes,
                    int t_begin, int t_end)
{
    const int nf = (int)p->freq.size(), nt = (int)p->lst.size(), K = p->n_basis, Kp = p->basis_Kp;
    const int np = p->basis_np;
    cpx<G> *grid = (cpx<G> *)wk.grid;
    cpx<G> *A = (cpx<G> *)wk.bufA, *Bb = (cpx<G> *)wk.bufB;
    G *frac = (G *)wk.frac;
    cpx<G> *cs = (cpx<G> *)wk.cs;
    const G *pre = (const G *)p->d_pre;
    const cpx<G> *tw = (const cpx<G> *)p->d_tw;
    const double es = sizeof(cpx<G>);
    const int nb = p->nbx * p->nby;
    const double nvis = 0.5 * p->n_src;
    const DimGeom *D = p->bg.dim;
    const size_t plane = (size_t)D[0].nf1 * D[1].nf1 * D[2].nf1;
    for (int t = t_begin; t < t_end; ++t) {
        TimeBin tb{};
        std::memcpy(tb.R, &p->Rt[(size_t)t * 9], 9 * sizeof(double));
        for (int i = 0; i < 3; ++i) {
            tb.C[i] = p->C[i];
            tb.qscale_top[i] = p->qscale_top[i];
            tb.nf1_top[i] = p->nf1_top[i];
        }
        tb.T[0] = p->T[0];
        tb.T[1] = p->T[1];
        tb.nbx = p->nbx;
        tb.nby = p->nby;
        CK(prof_begin(p, PC_BIN, st));
        CK(launch_time_binning(p->d_e, p->n_src, tb, wk.bin_of, wk.counts, wk.offsets, wk.cursor, wk.sdir, wk.sidx, nullptr,
                               st));
        CK(prof_end(p, (double)p->n_src * 80.0 + nb * 12.0));
        for (const auto &gr : p->groups) {
            if (gr.u1 <= gr.u0) continue;
            SliceGeom g = p->bg;
            std::memcpy(g.R, &p->Rt[(size_t)t * 9], 9 * sizeof(double));
            if (!p->beams.empty()) {
                g.beam = p->beams[gr.a];
                g.beam2 = p->beams[gr.b];
                g.two_beams = gr.a != gr.b;
            } else {
                g.two_beams = 0;
            }
            CK(prof_begin(p, PC_PREP, st));
            CK(launch_prep_basis<G>(wk.sdir, wk.sidx, wk.offsets + nb, p->n_src, p->d_bas_shat, (const G *)p->d_bas_Mg,
                                    (const G *)p->d_bas_dg, p->d_bas_freq, nf, K, Kp, g, wk.cell, frac, cs, st));
            CK(prof_end(p, nvis * (24.0 + 4.0 + K * 8.0 + 12.0 + 3.0 * sizeof(G) + Kp * es)));
            g.pre_x = pre + p->pre_off[0];                        // applied as the tile is stored
            g.pre_y = pre + p->pre_off[1];
            for (int k0 = 0; k0 < Kp; k0 += np) {
                CK(prof_begin(p, PC_SPREAD, st));
                CK(launch_spread_tile<G>(wk.offsets, wk.cell, frac, cs + (size_t)k0 * p->n_src, p->n_src, g, tb, 1.0,
                                         1.0, grid + (size_t)k0 * plane, st));
                CK(prof_end(p, nvis * (12.0 + 3.0 * sizeof(G) + np * es) + np * plane * es));
            }
            const long r1 = (long)K * D[2].nf1 * D[1].nf1;
            CK(prof_begin(p, PC_FFT_X, st));
            CK(launch_fft_pass<G>(grid, A, r1, D[0], nullptr, tw + p->tw_off[0], st));
            CK(prof_end(p, (double)r1 * (D[0].nf1 + D[0].B) * es));
            const long r2 = (long)D[0].B * K * D[2].nf1;
            CK(prof_begin(p, PC_FFT_Y, st));
            CK(launch_fft_pass<G>(A, Bb, r2, D[1], nullptr, tw + p->tw_off[1], st));
            CK(prof_end(p, (double)r2 * (D[1].nf1 + D[1].B) * es));
            const int nug = gr.u1 - gr.u0;
            CK(prof_begin(p, PC_INTERP, st));
            CK(launch_interp_basis<G>(Bb, gr.u0, nug, p->n_u, nf, (const G *)p->d_bas_Mg, K, p->d_bas_perm, p->d_bas_tm,
                                      (const G *)p->d_bas_tf, (const cpx<G> *)p->d_bas_ts, g, pre + p->pre_off[2],
                                      tw + p->tw_off[2], wk.Vu, st));
            // the K-plane band read once, each target's constants and perm entry, one FP64 complex out
            CK(prof_end(p, (double)D[1].B * D[0].B * K * D[2].nf1 * es +
                               (double)nug * nf * (16.0 + 4.0 + 4.0 * sizeof(G) + es + 16.0)));
        }
        CK(prof_begin(p, PC_SCATTER, st));
        CK(launch_scatter_basis(wk.Vu, p->d_bl2u, p->n_bl, p->n_u, nf, nt, t, vis, slice_bytes,
                                p->precision == FV_FP64, st));
        CK(prof_end(p, (double)p->n_bl * nf * (4 + 16.0) + (double)slice_bytes * nf));
    }
    return FV_OK;
}

template fv_status run_basis<float>(fv_plan_s *, fv_plan_s::Workspace &, cudaStream_t, char *, size_t, int, int);
template fv_status run_basis<double>(fv_plan_s *, fv_plan_s::Workspace &, cudaStream_t, char *, size_t, int, int);

cudaError_t refresh_flux_t(fv_plan_s *p, cudaStream_t st)
{
    if (!p->flux_borrowed || !p->d_flux_t || p->n_src == 0) return cudaSuccess;
    return launch_flux_transpose(p->flux, p->flux_fp64, p->n_src, p->n_stokes, (int)p->freq.size(), p->d_flux_t,
                                 st);
}

// The device status word after an execution: copied to pinned host memory behind the execution's work.
cudaError_t plan_post_status(fv_plan_s *p)
{
    cudaError_t e = cudaMemcpyAsync(p->h_status, p->d_status, sizeof(int), cudaMemcpyDeviceToHost, p->stream);
    if (e == cudaSuccess) e = cudaEventRecord(p->ev_status, p->stream);
    if (e == cudaSuccess) p->status_pending = true;
    return e;
}

// FV_ERR_TIMEOUT if a kernel of an earlier execution reported a bounded wait that ran out (its results
// were not valid), once; the word is then cleared.  wait: block until the last copy has landed, else
// look only if it already has.
fv_status plan_take_status(fv_plan_s *p, bool wait)
{
    if (!p->status_pending) return FV_OK;
    const cudaError_t q = wait ? cudaEventSynchronize(p->ev_status) : cudaEventQuery(p->ev_status);
    if (q == cudaErrorNotReady) return FV_OK;
    if (q != cudaSuccess) return p->fail(FV_ERR_CUDA, std::string("status event: ") + cudaGetErrorString(q));
    p->status_pending = false;
    if (*p->h_status == 0) return FV_OK;
    *p->h_status = 0;
    if (cudaMemsetAsync(p->d_status, 0, sizeof(int), p->stream) != cudaSuccess)
        return p->fail(FV_ERR_CUDA, "clearing the status word failed");
    return p->fail(FV_ERR_TIMEOUT, "a bounded wait in a kernel ran out; the results of that execution are invalid");
}

// All slices, t-major, split into contiguous chunks over the plan's streams
// (each with its own workspace); the streams fork from and join back to the
// plan's stream.
template <class G>
static fv_status execute_slices(fv_plan_s *p, char *vis, size_t slice_bytes, char *host_pinned)
{
    if ((int)p->ws.size() < p->n_streams) {
        // execution workspaces are allocated on first use (a plan run only through a batch never needs them)
        free_workspaces(p->ws);
        CK(alloc_workspaces(p->need, p->n_streams, p->ws));
    }
    // spectral-basis route: the unit of work is a time (all channels); the flux coefficients of this
    // execution's flux come first, on the plan's stream, before the fork
    const long total = p->use_basis ? (long)p->lst.size() : (long)p->freq.size() * p->lst.size();
    if (p->use_basis)
        CK(launch_basis_sky(p->flux, p->flux_fp64, p->n_src, (int)p->freq.size(), p->d_bas_M, p->n_basis,
                            p->d_bas_shat, p->stream));
    else if (p->flux_borrowed && p->d_flux_t) {
        // the channel-major flux copy from the borrowed buffer (read and written once)
        CK(prof_begin(p, PC_FLUX_T, p->stream));
        CK(refresh_flux_t(p, p->stream));
        CK(prof_end(p, 2.0 * p->n_src * p->n_stokes * p->freq.size() * (p->flux_fp64 ? 8 : 4)));
    }
    const int S = (int)std::min<long>(p->n_streams, std::max<long>(total, 1));
    if (S > 1) {
        CK(cudaEventRecord(p->ev_fork, p->stream));
        for (int s = 1; s < S; ++s) CK(cudaStreamWaitEvent(p->sub[s], p->ev_fork, 0));
    }
    for (int s = 0; s < S; ++s) {
        const long k0 = total * s / S, k1 = total * (s + 1) / S;
        OutMap om;
        om.host = host_pinned;
        fv_status st = p->use_basis ? run_basis<G>(p, p->ws[s], p->sub[s], vis, slice_bytes, (int)k0, (int)k1)
                                    : run_slices<G>(p, p->ws[s], p->sub[s], vis, slice_bytes, k0, k1, om);
        if (st != FV_OK) return st;
    }
    if (S > 1) {
        for (int s = 1; s < S; ++s) {
            CK(cudaEventRecord(p->ev_join[s], p->sub[s]));
            CK(cudaStreamWaitEvent(p->stream, p->ev_join[s], 0));
        }
    }
    return FV_OK;
}

extern "C" {

void fv_opts_default(fv_opts *o)
{
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->precision = FV_FP64;
    o->eps = 1e-10;
    o->beam = FV_BEAM_GAUSS;
    o->beam_param[0] = 10.0 * M_PI / 180.0;
    o->beam_param[1] = 150e6;
    o->upsampfac = 2.0;
    o->device = -1;
}

int fv_abi_version(void) { return FV_ABI_VERSION; }

int fv_lattice_detect(int n_ant, const double *enu_m, double tol_m, double basis[4], int *index)
{
    if (n_ant < 1 || !enu_m || !basis || !index) return 0;
    for (long i = 0; i < 3L * n_ant; ++i)
        if (!std::isfinite(enu_m[i])) return 0;
    return lattice_detect(n_ant, enu_m, tol_m, basis, index);
}

const char *fv_last_error(fv_plan_t p) { return p ? p->err.c_str() : g_create_error.c_str(); }

fv_status fv_plan(const fv_opts *o, fv_plan_t *out)
{
    if (!out) { g_create_error = "out is NULL"; return FV_ERR_ARG; }
    *out = nullptr;
    if (!o) { g_create_error = "opts is NULL"; return FV_ERR_ARG; }
    auto bad = [](const char *m) { g_create_error = m; return FV_ERR_ARG; };
    if (o->precision != FV_FP64 && o->precision != FV_MIXED) return bad("precision must be FV_FP64 or FV_MIXED");
    if (!(o->eps >= 1e-14 && o->eps <= 1e-2)) return bad("eps must be in [1e-14, 1e-2]");
    if (o->precision == FV_MIXED && o->eps < 1e-7) return bad("FV_MIXED needs eps >= 1e-7");
    if (o->n_freq < 1 || !o->freq_hz) return bad("need n_freq >= 1 and freq_hz");
    if (o->n_time < 1 || !o->lst_rad) return bad("need n_time >= 1 and lst_rad");
    for (int i = 0; i < o->n_freq; ++i)
        if (!(o->freq_hz[i] > 0.0) || !std::isfinite(o->freq_hz[i])) return bad("frequencies must be finite and > 0");
    for (int i = 0; i < o->n_time; ++i)
        if (!std::isfinite(o->lst_rad[i])) return bad("LSTs must be finite");
    if (!(std::fabs(o->latitude_rad) <= M_PI / 2)) return bad("latitude out of range");
    if (o->beam == FV_BEAM_GRID) return bad("a gridded beam is set by fv_set_beam_grid after fv_plan");
    if (o->beam < FV_BEAM_GAUSS || o->beam > FV_BEAM_UNIFORM) return bad("unknown beam");
    if (o->beam == FV_BEAM_GAUSS && !(o->beam_param[0] > 0 && o->beam_param[1] > 0))
        return bad("Gaussian beam needs FWHM > 0 and reference frequency > 0");
    if (o->beam == FV_BEAM_AIRY && !(o->beam_param[0] > 0)) return bad("Airy beam needs a diameter > 0");
    if (o->dims != 0 && o->dims != 2 && o->dims != 3) return bad("dims must be 0, 2 or 3");
    if (o->spread_method < FV_SPREAD_AUTO || o->spread_method > FV_SPREAD_TENSOR) return bad("unknown spread_method");
    if (o->bin_size[0] < 0 || o->bin_size[0] > 64 || o->bin_size[1] < 0 || o->bin_size[1] > 64)
        return bad("bin_size must be 0 or in [1, 64]");
    if (o->heights < FV_HEIGHTS_AUTO || o->heights > FV_HEIGHTS_TERMS) return bad("heights must be 0, 1 or 2");
    if (o->n_streams < 0) return bad("n_streams < 0");
    if (o->fft_max_radix != 0 && o->fft_max_radix != 8 && o->fft_max_radix != 16) return bad("fft_max_radix must be 0, 8 or 16");
    if (o->transform < FV_TRANSFORM_AUTO || o->transform > FV_TRANSFORM_BASIS) return bad("unknown transform");
    if (o->transform == FV_TRANSFORM_BASIS) {
        if (o->n_basis < 0 || o->n_basis > kBasisMax || o->n_basis > o->n_freq)
            return bad("the spectral-basis route needs 0 <= n_basis <= min(16, n_freq)");
        if (o->polarized) {
            g_create_error = "the spectral-basis route is defined for unpolarised skies (Appendix A)";
            return FV_ERR_UNSUPPORTED;
        }
    }
    if (o->transform == FV_TRANSFORM_LATTICE && o->dims == 3) return bad("the lattice route has no dims = 3 form");
    if (!(o->lattice_tol_m >= 0.0) || !std::isfinite(o->lattice_tol_m)) return bad("lattice_tol_m must be >= 0");
    double sigma = o->upsampfac == 0.0 ? 2.0 : o->upsampfac;
    if (!(sigma >= 1.25 && sigma <= 3.0)) return bad("upsampfac must be in [1.25, 3]");
    // the two deconvolutions amplify FP32 rounding by (Phihat(0)/Phihat(w pi/2 sigma))^2 at the band
    // edge: about 2e4 at sigma = 1.25 against 6 at sigma = 2, too much for FP32 spreading and FFTs
    if (o->precision == FV_MIXED && sigma < 1.5) return bad("FV_MIXED needs upsampfac >= 1.5");
    int w = o->kernel_width;
    if (w == 0) {
        if (std::fabs(sigma - 2.0) < 1e-12)
            w = (int)std::ceil(std::log10(1.0 / o->eps) - 1e-12) + 1;   // Section 2.2 rule at sigma = 2
        else
            // the estimate eps ~ exp(-pi w sqrt(1 - 1/sigma)) of the kernel's aliasing error, plus a margin
            // of two points: the type-3 transform applies the kernel twice and divides by its transform twice
            w = (int)std::ceil(std::log(1.0 / o->eps) / (M_PI * std::sqrt(1.0 - 1.0 / sigma)) - 1e-12) + 2;
        w = std::max(2, w);
        if (w > 16) {
            // a narrower kernel would miss eps: refuse rather than return a less accurate result
            g_create_error = "eps " + std::to_string(o->eps) + " at upsampfac " + std::to_string(sigma) +
                             " needs a kernel width of " + std::to_string(w) + " (at most 16)";
            return FV_ERR_UNSUPPORTED;
        }
    }
    if (w < 2 || w > 16) return bad("kernel_width must be in [2, 16]");

    int ndev = 0;
    cudaError_t ce = cudaGetDeviceCount(&ndev);
    if (ce != cudaSuccess || ndev < 1) {
        g_create_error = std::string("no usable CUDA device: ") + cudaGetErrorString(ce);
        cudaGetLastError();
        return FV_ERR_CUDA;
    }
    int dev = o->device;
    if (dev < 0) {
        if (cudaGetDevice(&dev) != cudaSuccess) dev = 0;
    }
    if (dev >= ndev) return bad("device ordinal out of range");
    if (cudaSetDevice(dev) != cudaSuccess) { g_create_error = "cudaSetDevice failed"; return FV_ERR_CUDA; }

    fv_plan_s *p = new (std::nothrow) fv_plan_s();
    if (!p) { g_create_error = "host allocation failed"; return FV_ERR_OOM; }
    p->precision = o->precision;
    p->eps = o->eps;
    p->freq.assign(o->freq_hz, o->freq_hz + o->n_freq);
    p->lst.assign(o->lst_rad, o->lst_rad + o->n_time);
    p->lat = o->latitude_rad;
    p->beam.kind = o->beam;
    p->beam.p0 = o->beam_param[0];
    p->beam.p1 = o->beam_param[1];
    p->beam.p2 = o->beam_param[2];
    beam_float_constant(p->beam);
    p->polarized = o->polarized ? 1 : 0;
    p->n_pol = p->polarized ? 4 : 1;
    p->dims_req = o->dims;
    p->sigma = sigma;
    p->w = w;
    p->beta = 2.30 * w * (1.0 - 1.0 / (2.0 * sigma)) / 0.75;   // 2.3 w at sigma = 2 (Section 2.2)
    p->device = dev;
    if (o->cuda_stream) {
        p->stream = (cudaStream_t)o->cuda_stream;
    } else {
        if (cudaStreamCreateWithFlags(&p->stream, cudaStreamNonBlocking) != cudaSuccess) {
            delete p;
            g_create_error = "cudaStreamCreate failed";
            return FV_ERR_CUDA;
        }
        p->own_stream = true;
    }
    // execution streams: sub[0] is the plan's stream, the others are owned by the plan
    // measured on one GB300 (127-antenna workload): slices gain from 8 concurrent streams (type-3 +4 %,
    // lattice +15 % over 4); a spectral-basis time fills the GPU alone, so more streams would only hold
    // more ~1 GB workspaces
    p->n_streams = o->n_streams > 0 ? std::min(o->n_streams, 16) : (o->transform == FV_TRANSFORM_BASIS ? 4 : 8);
    p->spread_req = o->spread_method;
    p->bin_req[0] = o->bin_size[0];
    p->bin_req[1] = o->bin_size[1];
    p->heights_req = o->heights;
    // radix 8 needs fewer registers (more CTAs per SM), which wins in FP32; FP64 uses the same
    // register count either way and prefers fewer stages
    p->fft_max_radix = o->fft_max_radix > 0 ? o->fft_max_radix : 16;
    p->transform_req = o->transform;
    p->use_basis = o->transform == FV_TRANSFORM_BASIS;
    p->n_basis_req = p->use_basis ? o->n_basis : 0;
    p->n_basis = p->n_basis_req;
    p->lat_tol = o->lattice_tol_m > 0.0 ? o->lattice_tol_m : 1e-10;
    p->sub.assign(p->n_streams, nullptr);
    p->ev_join.assign(p->n_streams, nullptr);
    p->sub[0] = p->stream;
    bool ok = cudaEventCreateWithFlags(&p->ev_fork, cudaEventDisableTiming) == cudaSuccess;
    for (int s = 1; s < p->n_streams && ok; ++s) {
        ok = cudaStreamCreateWithFlags(&p->sub[s], cudaStreamNonBlocking) == cudaSuccess &&
             cudaEventCreateWithFlags(&p->ev_join[s], cudaEventDisableTiming) == cudaSuccess;
    }
    if (!ok) {
        g_create_error = "stream or event creation failed";
        fv_destroy(p);
        return FV_ERR_CUDA;
    }
    // rotation matrices, equatorial -> ENU (Section 2.3 rigid rotation)
    p->Rt.resize((size_t)o->n_time * 9);
    const double sphi = std::sin(p->lat), cphi = std::cos(p->lat);
    for (int t = 0; t < o->n_time; ++t) {
        double sl = std::sin(p->lst[t]), cl = std::cos(p->lst[t]);
        double *R = &p->Rt[(size_t)t * 9];
        R[0] = -sl;         R[1] = cl;          R[2] = 0.0;
        R[3] = -sphi * cl;  R[4] = -sphi * sl;  R[5] = cphi;
        R[6] = cphi * cl;   R[7] = cphi * sl;   R[8] = sphi;
    }
    // quadrature nodes for Phihat: z = sin(pi x / 2) removes the sqrt edge
    p->nq = 4 * w + 40;
    std::vector<double> gx, gw;
    gauss_legendre(p->nq, gx, gw);
    std::vector<double> zx(p->nq), zw(p->nq);
    for (int q = 0; q < p->nq; ++q) {
        double th = 0.5 * M_PI * gx[q];
        zx[q] = std::sin(th);
        zw[q] = 0.5 * M_PI * gw[q] * std::cos(th);
    }
    fv_status s = FV_OK;
    if (cudaMalloc(&p->d_glx, p->nq * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&p->d_glw, p->nq * sizeof(double)) != cudaSuccess ||
        cudaMemcpy(p->d_glx, zx.data(), p->nq * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(p->d_glw, zw.data(), p->nq * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMalloc(&p->d_status, sizeof(int)) != cudaSuccess || cudaMemset(p->d_status, 0, sizeof(int)) != cudaSuccess ||
        cudaMallocHost(&p->h_status, sizeof(int)) != cudaSuccess ||
        cudaEventCreateWithFlags(&p->ev_status, cudaEventDisableTiming) != cudaSuccess)
        s = FV_ERR_CUDA;
    if (p->h_status) *p->h_status = 0;
    if (s != FV_OK) {
        g_create_error = "device set-up failed";
        fv_destroy(p);
        return s;
    }
    *out = p;
    return FV_OK;
}

// Baselines, unique targets, beam groups, lattice test and device tables from the stored array
// (p->enu_h, p->pairs_h) and beams.
static fv_status setup_array(fv_plan_s *p)
{
    const int n_ant = (int)(p->enu_h.size() / 3), n_bl = (int)(p->pairs_h.size() / 2);
    const double *enu_m = p->enu_h.data();
    const std::vector<int> &pr = p->pairs_h;
    const bool multi = !p->beams.empty();
    // beam groups: unordered pairs of beam indices, in increasing order
    auto pair_of = [&](int b) {
        int ba = multi ? p->beam_of_ant[pr[2 * b]] : 0, bb = multi ? p->beam_of_ant[pr[2 * b + 1]] : 0;
        return std::make_pair(std::min(ba, bb), std::max(ba, bb));
    };
    std::map<std::pair<int, int>, int> gid;
    for (int b = 0; b < n_bl; ++b) gid.emplace(pair_of(b), 0);
    std::vector<fv_plan_s::BeamGroup> groups;
    for (auto &kv : gid) {
        kv.second = (int)groups.size();
        fv_plan_s::BeamGroup g;
        g.a = kv.first.first;
        g.b = kv.first.second;
        groups.push_back(g);
    }
    std::vector<int> grp_of(n_bl, 0);
    for (int b = 0; b < n_bl; ++b) grp_of[b] = gid[pair_of(b)];
    // baselines by group; unique baseline vectors within a group, bit-exact (Fig. 1, panel E), numbered
    // group by group so that every group's targets are contiguous
    std::vector<int> grp_bl;
    std::vector<double> bu;
    std::vector<int> bl2u(n_bl);
    bool nonplanar = false;
    for (size_t g = 0; g < groups.size(); ++g) {
        groups[g].bl0 = (int)grp_bl.size();
        groups[g].u0 = (int)(bu.size() / 3);
        std::map<std::tuple<double, double, double>, int> uid;
        for (int b = 0; b < n_bl; ++b) {
            if (grp_of[b] != (int)g) continue;
            grp_bl.push_back(b);
            const double *xi = enu_m + 3 * pr[2 * b], *xj = enu_m + 3 * pr[2 * b + 1];
            double v[3] = {xi[0] - xj[0], xi[1] - xj[1], xi[2] - xj[2]};
            if (v[2] != 0.0) nonplanar = true;
            auto key = std::make_tuple(v[0] + 0.0, v[1] + 0.0, v[2] + 0.0);   // +0.0 folds -0 into 0
            auto it = uid.find(key);
            if (it == uid.end()) {
                int id = (int)(bu.size() / 3);
                uid.emplace(key, id);
                bu.insert(bu.end(), v, v + 3);
                bl2u[b] = id;
            } else {
                bl2u[b] = it->second;
            }
        }
        groups[g].bl1 = (int)grp_bl.size();
        groups[g].u1 = (int)(bu.size() / 3);
    }
    if (groups.empty()) groups.push_back(fv_plan_s::BeamGroup{});
    int d = p->dims_req ? p->dims_req : (nonplanar ? 3 : 2);
    if (d == 2 && nonplanar) return p->fail(FV_ERR_ARG, "dims = 2 requested for a non-coplanar array");
    // lattice test (Section 2.2.1): baselines as integer combinations n of two lattice vectors
    std::vector<int> bln;
    bool lat_ok = false;
    double lat_basis[4] = {0, 0, 0, 0};
    int lat_H[2] = {0, 0};
    if (n_ant <= 20000) {      // the test is O(n_ant^2) on the host
        std::vector<int> kidx(2 * (size_t)n_ant);
        lat_ok = lattice_detect(n_ant, enu_m, p->lat_tol, lat_basis, kidx.data()) != 0;
        if (lat_ok) {
            p->lat_bup.resize(n_bl);
            for (int b = 0; b < n_bl; ++b) p->lat_bup[b] = enu_m[3 * pr[2 * b] + 2] - enu_m[3 * pr[2 * b + 1] + 2];
            bln.resize(2 * (size_t)n_bl);
            for (int b = 0; b < n_bl; ++b)
                for (int k = 0; k < 2; ++k) {
                    const int v = kidx[2 * pr[2 * b] + k] - kidx[2 * pr[2 * b + 1] + k];
                    bln[2 * b + k] = v;
                    lat_H[k] = std::max(lat_H[k], std::abs(v));
                }
        }
    }
    if (p->transform_req == FV_TRANSFORM_LATTICE && !lat_ok)
        return p->fail(FV_ERR_UNSUPPORTED, "transform = FV_TRANSFORM_LATTICE, but the antennas' horizontal "
                                           "positions are not a lattice within lattice_tol_m");
    if (!lat_ok) p->lat_bup.clear();
    p->lat_ok = lat_ok;        // reported whatever the route; the lattice route also needs transform != TYPE3
                               // and dims != 3
    std::memcpy(p->lat_basis, lat_basis, sizeof(lat_basis));
    p->lat_H[0] = lat_H[0];
    p->lat_H[1] = lat_H[1];
    p->n_ant = n_ant;
    p->n_bl = n_bl;
    p->n_u = (int)(bu.size() / 3);
    p->d = d;
    p->d_array = d;
    p->hK = 0;
    p->bu.swap(bu);
    p->bl2u.swap(bl2u);
    p->groups.swap(groups);
    for (int i = 0; i < 3; ++i) {
        double lo = INFINITY, hi = -INFINITY;
        for (int u = 0; u < p->n_u; ++u) { lo = std::min(lo, p->bu[3 * u + i]); hi = std::max(hi, p->bu[3 * u + i]); }
        if (p->n_u == 0) lo = hi = 0.0;
        p->bcen[i] = 0.5 * (lo + hi);
        p->bhalf[i] = 0.5 * (hi - lo);
    }
    dfree_t(p->d_bu);
    dfree_t(p->d_dec);
    dfree_t(p->d_tgt_db);
    dfree_t(p->d_tgt_bc);
    p->tgt_n = 0;
    dfree_t(p->d_bl2u);
    dfree_t(p->d_u_off);
    dfree_t(p->d_u_bl);
    dfree_t(p->d_bln);
    dfree_t(p->d_grp_bl);
    if (lat_ok) {
        CK(cudaMalloc(&p->d_bln, std::max<size_t>(bln.size(), 2) * sizeof(int)));
        if (!bln.empty())
            CK(cudaMemcpyAsync(p->d_bln, bln.data(), bln.size() * sizeof(int), cudaMemcpyHostToDevice, p->stream));
    }
    const size_t nu = std::max(p->n_u, 1), nb = std::max(p->n_bl, 1);
    CK(cudaMalloc(&p->d_bu, nu * 3 * sizeof(double)));
    CK(cudaMalloc(&p->d_dec, nu * sizeof(double)));
    CK(cudaMalloc(&p->d_bl2u, nb * sizeof(int)));
    CK(cudaMalloc(&p->d_grp_bl, nb * sizeof(int)));
    if (p->n_u) CK(cudaMemcpyAsync(p->d_bu, p->bu.data(), (size_t)p->n_u * 3 * sizeof(double), cudaMemcpyHostToDevice, p->stream));
    {
        // CSR of the baselines of every unique target (counting sort of bl2u)
        std::vector<int> u_off((size_t)p->n_u + 1, 0), u_bl(std::max(p->n_bl, 1), 0);
        for (int b = 0; b < p->n_bl; ++b) ++u_off[(size_t)p->bl2u[b] + 1];
        for (int u = 0; u < p->n_u; ++u) u_off[(size_t)u + 1] += u_off[u];
        std::vector<int> cur(u_off.begin(), u_off.end() - 1);
        for (int b = 0; b < p->n_bl; ++b) u_bl[(size_t)cur[p->bl2u[b]]++] = b;
        CK(cudaMalloc(&p->d_u_off, u_off.size() * sizeof(int)));
        CK(cudaMalloc(&p->d_u_bl, u_bl.size() * sizeof(int)));
        CK(cudaMemcpy(p->d_u_off, u_off.data(), u_off.size() * sizeof(int), cudaMemcpyHostToDevice));
        CK(cudaMemcpy(p->d_u_bl, u_bl.data(), u_bl.size() * sizeof(int), cudaMemcpyHostToDevice));
    }
    if (p->n_bl) {
        CK(cudaMemcpyAsync(p->d_bl2u, p->bl2u.data(), (size_t)p->n_bl * sizeof(int), cudaMemcpyHostToDevice, p->stream));
        CK(cudaMemcpyAsync(p->d_grp_bl, grp_bl.data(), (size_t)p->n_bl * sizeof(int), cudaMemcpyHostToDevice,
                           p->stream));
    }
    CK(launch_target_deconv(p->d_bu, p->n_u, p->d, p->bcen, p->bhalf, p->w, p->beta, p->sigma, p->d_glx, p->d_glw,
                            p->nq, p->d_dec, p->stream));
    p->dec_d = p->d;
    CK(cudaStreamSynchronize(p->stream));
    p->have_array = true;
    if (p->have_sky) return prepare(p);
    return FV_OK;
}


fv_status fv_set_array(fv_plan_t p, int n_ant, const double *enu_m, int n_bl, const int *pairs)
{
    if (p) ++p->gen;
    if (!p) return FV_ERR_ARG;
    if (cudaSetDevice(p->device) != cudaSuccess) return p->fail(FV_ERR_CUDA, "cudaSetDevice failed");
    if (n_ant < 1 || !enu_m) return p->fail(FV_ERR_ARG, "need n_ant >= 1 and positions");
    for (long i = 0; i < 3L * n_ant; ++i)
        if (!std::isfinite(enu_m[i])) return p->fail(FV_ERR_ARG, "non-finite antenna position");
    std::vector<int> pr;
    if (pairs) {
        if (n_bl < 0) return p->fail(FV_ERR_ARG, "n_bl < 0");
        pr.assign(pairs, pairs + 2L * n_bl);
        for (int v : pr)
            if (v < 0 || v >= n_ant) return p->fail(FV_ERR_ARG, "antenna index out of range");
    } else {
        for (int i = 0; i < n_ant; ++i)
            for (int j = i + 1; j < n_ant; ++j) { pr.push_back(i); pr.push_back(j); }
    }
    if (!p->beams.empty() && (int)p->beam_of_ant.size() != n_ant) {
        // per-antenna beams set for another array: back to the shared beam
        p->beams.clear();
        p->beam_of_ant.clear();
    }
    p->enu_h.assign(enu_m, enu_m + 3L * n_ant);
    p->pairs_h.swap(pr);
    return setup_array(p);
}

fv_status fv_set_beams(fv_plan_t p, int n_beams, const int *kinds, const double *params, const int *beam_of_ant)
{
    if (p) ++p->gen;
    if (!p) return FV_ERR_ARG;
    if (cudaSetDevice(p->device) != cudaSuccess) return p->fail(FV_ERR_CUDA, "cudaSetDevice failed");
    if (!p->have_array) return p->fail(FV_ERR_STATE, "fv_set_array must come before fv_set_beams");
    if (n_beams <= 0 || !beam_of_ant) {
        drop_beam_grids(p);
        p->beams.clear();
        p->beam_of_ant.clear();
        return setup_array(p);
    }
    if (n_beams > 16) return p->fail(FV_ERR_ARG, "at most 16 beams");
    if (!kinds || !params) return p->fail(FV_ERR_ARG, "NULL beam kinds or parameters");
    std::vector<BeamParams> beams(n_beams);
    for (int k = 0; k < n_beams; ++k) {
        const double *q = params + 3 * k;
        if (kinds[k] < FV_BEAM_GAUSS || kinds[k] > FV_BEAM_UNIFORM) return p->fail(FV_ERR_ARG, "unknown beam kind");
        if (kinds[k] == FV_BEAM_GAUSS && !(q[0] > 0 && q[1] > 0))
            return p->fail(FV_ERR_ARG, "Gaussian beam needs FWHM > 0 and reference frequency > 0");
        if (kinds[k] == FV_BEAM_AIRY && !(q[0] > 0)) return p->fail(FV_ERR_ARG, "Airy beam needs a diameter > 0");
        beams[k].kind = kinds[k];
        beams[k].p0 = q[0];
        beams[k].p1 = q[1];
        beams[k].p2 = q[2];
        beam_float_constant(beams[k]);
    }
    std::vector<int> boa(beam_of_ant, beam_of_ant + p->n_ant);
    for (int v : boa)
        if (v < 0 || v >= n_beams) return p->fail(FV_ERR_ARG, "beam index out of range");
    drop_beam_grids(p);
    p->beams.swap(beams);
    p->beam_of_ant.swap(boa);
    return setup_array(p);
}

// Cubic B-spline coefficients c of samples f along one axis, c[i-1] + 4 c[i] + c[i+1] = 6 f[i]:
// with the out-of-range knots mirrored about the end samples (Thomas algorithm; rows 0 and n-1 carry a
// 2 for the mirrored neighbour), or wrapped (cyclic tridiagonal, Sherman-Morrison).  In place,
// elements f[k * stride], k < n.
static void bspline_prefilter(double *f, int n, long stride, bool periodic)
{
    if (n == 1) return;
    std::vector<double> r(n), x(n);
    for (int k = 0; k < n; ++k) r[k] = 6.0 * f[k * stride];
    if (n == 2) {
        // both boundary rules give 4 c0 + 2 c1 = r0, 2 c0 + 4 c1 = r1
        x[0] = (4.0 * r[0] - 2.0 * r[1]) / 12.0;
        x[1] = (4.0 * r[1] - 2.0 * r[0]) / 12.0;
    } else if (!periodic) {
        std::vector<double> cp(n), dp(n);
        // row 0: 4 c0 + 2 c1; rows 1..n-2: c_{k-1} + 4 c_k + c_{k+1}; row n-1: 2 c_{n-2} + 4 c_{n-1}
        cp[0] = 2.0 / 4.0;
        dp[0] = r[0] / 4.0;
        for (int k = 1; k < n; ++k) {
            const double a = k == n - 1 ? 2.0 : 1.0, c = k == n - 1 ? 0.0 : 1.0;
            const double m = 4.0 - a * cp[k - 1];
            cp[k] = c / m;
            dp[k] = (r[k] - a * dp[k - 1]) / m;
        }
        x[n - 1] = dp[n - 1];
        for (int k = n - 2; k >= 0; --k) x[k] = dp[k] - cp[k] * x[k + 1];
    } else {
        // A = tridiag(1, 4, 1) with corners 1 = B + u v^T, u = (g, 0.., 1), v = (1, 0.., 1/g), g = -4
        const double g = -4.0;
        auto thomas = [&](std::vector<double> &rhs, std::vector<double> &out) {
            std::vector<double> cp(n), dp(n);
            double b0 = 4.0 - g;
            cp[0] = 1.0 / b0;
            dp[0] = rhs[0] / b0;
            for (int k = 1; k < n; ++k) {
                const double b = k == n - 1 ? 4.0 - 1.0 / g : 4.0;
                const double m = b - cp[k - 1];
                cp[k] = 1.0 / m;
                dp[k] = (rhs[k] - dp[k - 1]) / m;
            }
            out[n - 1] = dp[n - 1];
            for (int k = n - 2; k >= 0; --k) out[k] = dp[k] - cp[k] * out[k + 1];
        };
        std::vector<double> u(n, 0.0), z(n);
        u[0] = g;
        u[n - 1] = 1.0;
        thomas(r, x);
        thomas(u, z);
        const double fact = (x[0] + x[n - 1] / g) / (1.0 + z[0] + z[n - 1] / g);
        for (int k = 0; k < n; ++k) x[k] -= fact * z[k];
    }
    for (int k = 0; k < n; ++k) f[k * stride] = x[k];
}

fv_status fv_set_beam_grid(fv_plan_t p, int beam, int n_theta, int n_phi, int order, const double *voltage)
{
    if (p) ++p->gen;
    if (!p) return FV_ERR_ARG;
    if (cudaSetDevice(p->device) != cudaSuccess) return p->fail(FV_ERR_CUDA, "cudaSetDevice failed");
    if (beam < -1 || beam >= (int)p->beams.size())
        return p->fail(FV_ERR_ARG, "beam index out of range (per-antenna beams come from fv_set_beams)");
    if (n_theta < 2 || n_phi < 1 || (long)n_theta * n_phi > (1L << 22))
        return p->fail(FV_ERR_ARG, "need n_theta >= 2, n_phi >= 1 and n_theta * n_phi <= 2^22");
    if (order != 1 && order != 3) return p->fail(FV_ERR_ARG, "interpolation order must be 1 or 3");
    if (!voltage) return p->fail(FV_ERR_ARG, "NULL beam samples");
    const size_t n = p->freq.size() * (size_t)n_theta * n_phi;
    for (size_t i = 0; i < n; ++i)
        if (!std::isfinite(voltage[i])) return p->fail(FV_ERR_ARG, "non-finite beam sample");
    std::vector<double> table;
    if (order == 3) {
        // bicubic: the B-spline coefficients of every channel's plane, zenith-angle columns then
        // azimuth rows
        table.assign(voltage, voltage + n);
        for (size_t f = 0; f < p->freq.size(); ++f) {
            double *pl = table.data() + f * (size_t)n_theta * n_phi;
            for (int j = 0; j < n_phi; ++j) bspline_prefilter(pl + j, n_theta, n_phi, false);
            for (int i = 0; i < n_theta; ++i) bspline_prefilter(pl + (size_t)i * n_phi, n_phi, 1, true);
        }
        voltage = table.data();
    }
    const bool fp64 = p->precision == FV_FP64;
    void *d = nullptr;
    CK(cudaMalloc(&d, n * (fp64 ? sizeof(double) : sizeof(float))));
    cudaError_t e;
    if (fp64) {
        e = cudaMemcpy(d, voltage, n * sizeof(double), cudaMemcpyHostToDevice);
    } else {
        std::vector<float> v32(voltage, voltage + n);
        e = cudaMemcpy(d, v32.data(), n * sizeof(float), cudaMemcpyHostToDevice);
    }
    if (e != cudaSuccess) {
        cudaFree(d);
        return p->fail(FV_ERR_CUDA, cudaGetErrorString(e));
    }
    if (beam < 0) {
        dfree(p->d_grid_main);
        p->d_grid_main = d;
    } else {
        p->d_grid_beams.resize(p->beams.size(), nullptr);
        dfree(p->d_grid_beams[beam]);
        p->d_grid_beams[beam] = d;
    }
    BeamParams &b = beam < 0 ? p->beam : p->beams[beam];
    b.kind = FV_BEAM_GRID;
    b.grid = d;
    b.grid_fp64 = fp64 ? 1 : 0;
    b.n_th = n_theta;
    b.n_ph = n_phi;
    b.grid_order = order;
    // the slices' geometry holds copies of the plan's beam
    for (auto &g : p->gf) g.beam = p->beam;
    p->bg.beam = p->beam;
    return FV_OK;
}

fv_status fv_set_sky(fv_plan_t p, long n_src, const double *ra_rad, const double *dec_rad, int n_stokes,
                     const void *flux, int flux_is_fp64, int flux_on_device)
{
    if (p) ++p->gen;
    if (!p) return FV_ERR_ARG;
    if (cudaSetDevice(p->device) != cudaSuccess) return p->fail(FV_ERR_CUDA, "cudaSetDevice failed");
    if (!p->have_array) return p->fail(FV_ERR_STATE, "fv_set_array must come before fv_set_sky");
    if (n_src < 0) return p->fail(FV_ERR_ARG, "n_src < 0");
    if (n_stokes != (p->polarized ? 4 : 1) && !(n_stokes == 4 && !p->polarized))
        return p->fail(FV_ERR_ARG, p->polarized ? "polarised plan needs n_stokes = 4" : "n_stokes must be 1 or 4");
    if (n_src > 0 && (!ra_rad || !dec_rad || !flux)) return p->fail(FV_ERR_ARG, "NULL sky array");
    for (long i = 0; i < n_src; ++i)
        if (!std::isfinite(ra_rad[i]) || !std::isfinite(dec_rad[i]))
            return p->fail(FV_ERR_ARG, "non-finite source coordinate");
    p->have_sky = false;
    // work still queued on the device may read the sky buffers this call rewrites (a plan's own streams,
    // or a batch's lanes): wait for it, as freeing them would
    CK(cudaDeviceSynchronize());
    // (re)allocate a buffer only when its size changes
    auto ensure = [&](void **ptr, size_t &cap, size_t bytes) -> cudaError_t {
        if (*ptr && cap == bytes) return cudaSuccess;
        if (*ptr) cudaFree(*ptr);
        *ptr = nullptr;
        cap = 0;
        cudaError_t e = cudaMalloc(ptr, bytes);
        if (e == cudaSuccess) cap = bytes;
        return e;
    };
    p->flux = nullptr;
    p->flux_borrowed = false;
    p->n_src = n_src;
    p->n_stokes = n_stokes;
    p->flux_fp64 = flux_is_fp64 ? 1 : 0;
    const size_t ns = std::max<long>(n_src, 1);
    CK(ensure((void **)&p->d_e, p->e_bytes, ns * 3 * sizeof(double)));
    CK(ensure((void **)&p->d_radec, p->radec_bytes, ns * 2 * sizeof(double)));
    double *d_tmp = p->d_radec;
    if (n_src) {
        CK(cudaMemcpyAsync(d_tmp, ra_rad, n_src * sizeof(double), cudaMemcpyHostToDevice, p->stream));
        CK(cudaMemcpyAsync(d_tmp + ns, dec_rad, n_src * sizeof(double), cudaMemcpyHostToDevice, p->stream));
    }
    CK(launch_radec_to_unit(d_tmp, d_tmp + ns, n_src, p->d_e, p->stream));
    const size_t fbytes = (size_t)n_stokes * n_src * p->freq.size() * (p->flux_fp64 ? 8 : 4);
    if (flux_on_device) {
        p->flux = flux;
        p->flux_borrowed = true;
        dfree(p->d_flux_owned);
        p->flux_owned_bytes = 0;
    } else if (n_src) {
        CK(ensure(&p->d_flux_owned, p->flux_owned_bytes, fbytes));
        CK(cudaMemcpyAsync(p->d_flux_owned, flux, fbytes, cudaMemcpyHostToDevice, p->stream));
        p->flux = p->d_flux_owned;
    }
    if (n_src && !p->use_basis) {
        // the channel-major copy the slices read: made now from an owned copy, at every execution from a
        // borrowed buffer
        CK(ensure(&p->d_flux_t, p->flux_t_bytes, fbytes));
        if (!p->flux_borrowed)
            CK(launch_flux_transpose(p->flux, p->flux_fp64, n_src, n_stokes, (int)p->freq.size(), p->d_flux_t,
                                     p->stream));
    }
    // source extents over all times (visible directions only)
    const int nb = 304;
    if (!p->d_Rt) CK(cudaMalloc(&p->d_Rt, std::max<size_t>(p->Rt.size(), 1) * sizeof(double)));
    if (!p->d_ext) CK(cudaMalloc(&p->d_ext, (size_t)nb * 6 * sizeof(double)));
    double *d_R = p->d_Rt, *d_ext = p->d_ext;
    CK(cudaMemcpyAsync(d_R, p->Rt.data(), p->Rt.size() * sizeof(double), cudaMemcpyHostToDevice, p->stream));
    CK(launch_source_extents(p->d_e, n_src, d_R, (int)p->lst.size(), d_ext, nb, p->stream));
    std::vector<double> ext((size_t)nb * 6);
    CK(cudaMemcpyAsync(ext.data(), d_ext, ext.size() * sizeof(double), cudaMemcpyDeviceToHost, p->stream));
    CK(cudaStreamSynchronize(p->stream));
    (void)d_tmp;
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int b = 0; b < nb; ++b)
        for (int i = 0; i < 3; ++i) {
            lo[i] = std::min(lo[i], ext[(size_t)b * 6 + i]);
            hi[i] = std::max(hi[i], ext[(size_t)b * 6 + 3 + i]);
        }
    p->any_visible = std::isfinite(lo[0]);
    for (int i = 0; i < 3; ++i) {
        if (p->any_visible) {
            p->C[i] = 0.5 * (lo[i] + hi[i]);
            p->S[i] = 0.5 * (hi[i] - lo[i]);
        } else {
            p->C[i] = 0.0;
            p->S[i] = 0.0;
        }
    }
    fv_status s = prepare(p);
    if (s != FV_OK) return s;
    p->have_sky = true;
    return FV_OK;
}

fv_status fv_execute(fv_plan_t p, void *vis, int vis_on_device)
{
    if (!p) return FV_ERR_ARG;
    if (!vis) return p->fail(FV_ERR_ARG, "vis is NULL");
    if (!p->have_array || !p->have_sky) return p->fail(FV_ERR_STATE, "fv_set_array and fv_set_sky must come first");
    if (cudaSetDevice(p->device) != cudaSuccess) return p->fail(FV_ERR_CUDA, "cudaSetDevice failed");
    const size_t cb = p->precision == FV_FP64 ? 16 : 8;
    if (vis_on_device && (uintptr_t)vis % cb != 0)
        return p->fail(FV_ERR_ARG, "vis must be aligned to its element size (" + std::to_string(cb) + " bytes)");
    fv_status prev = plan_take_status(p, false);
    if (prev != FV_OK) return prev;
    const size_t slice_bytes = (size_t)p->n_bl * p->n_pol * cb;
    const size_t total = slice_bytes * p->freq.size() * p->lst.size();
    char *dst = (char *)vis;
    void *tmp = nullptr;
    // host output in pinned memory: every slice is copied out as soon as it is written (the slice routes),
    // overlapping the copies with the other slices' kernels; pageable memory gets one copy at the end
    char *host_pinned = nullptr;
    if (!vis_on_device) {
        CK(cudaMallocAsync(&tmp, std::max<size_t>(total, 1), p->stream));
        dst = (char *)tmp;
        cudaPointerAttributes pa{};
        if (cudaPointerGetAttributes(&pa, vis) == cudaSuccess && pa.type == cudaMemoryTypeHost && !p->use_basis)
            host_pinned = (char *)vis;
        cudaGetLastError();
    }
    fv_status s;
    if (!p->any_visible || p->n_src == 0) {
        CK(cudaMemsetAsync(dst, 0, total, p->stream));
        host_pinned = nullptr;
        s = FV_OK;
    } else {
        s = p->precision == FV_FP64 ? execute_slices<double>(p, dst, slice_bytes, host_pinned)
                                    : execute_slices<float>(p, dst, slice_bytes, host_pinned);
    }
    if (s == FV_OK) CK(plan_post_status(p));
    if (!vis_on_device) {
        if (s == FV_OK && !host_pinned) CK(cudaMemcpyAsync(vis, tmp, total, cudaMemcpyDeviceToHost, p->stream));
        cudaFreeAsync(tmp, p->stream);
        CK(cudaStreamSynchronize(p->stream));
        if (s == FV_OK) s = plan_take_status(p, true);
    }
    return s;
}

fv_status fv_destroy(fv_plan_t p)
{
    if (!p) return FV_OK;
    cudaSetDevice(p->device);
    for (cudaStream_t st : p->sub)
        if (st) cudaStreamSynchronize(st);
    if (p->stream) cudaStreamSynchronize(p->stream);
    free_geometry(p);
    dfree_t(p->d_glx);
    dfree_t(p->d_glw);
    dfree_t(p->d_bu);
    dfree_t(p->d_dec);
    dfree_t(p->d_tgt_db);
    dfree_t(p->d_tgt_bc);
    p->tgt_n = 0;
    dfree_t(p->d_bl2u);
    dfree_t(p->d_u_off);
    dfree_t(p->d_u_bl);
    dfree_t(p->d_bln);
    dfree_t(p->d_grp_bl);
    dfree_t(p->d_e);
    dfree(p->d_flux_owned);
    dfree(p->d_flux_t);
    dfree_t(p->d_radec);
    dfree_t(p->d_Rt);
    dfree_t(p->d_ext);
    dfree(p->d_grid_main);
    dfree_t(p->d_status);
    if (p->h_status) cudaFreeHost(p->h_status);
    if (p->ev_status) cudaEventDestroy(p->ev_status);
    drop_beam_grids(p);
    for (cudaEvent_t ev : p->ev_pool) cudaEventDestroy(ev);
    for (size_t s = 1; s < p->sub.size(); ++s) {
        if (p->sub[s]) cudaStreamDestroy(p->sub[s]);
        if (p->ev_join[s]) cudaEventDestroy(p->ev_join[s]);
    }
    if (p->ev_fork) cudaEventDestroy(p->ev_fork);
    if (p->own_stream && p->stream) cudaStreamDestroy(p->stream);
    delete p;
    return FV_OK;
}

fv_status fv_get_info(fv_plan_t p, fv_info *info)
{
    if (!p || !info) return FV_ERR_ARG;
    std::memset(info, 0, sizeof(*info));
    info->dims = p->use_lattice ? p->d_array : p->d;
    info->kernel_width = p->w;
    info->beta = p->beta;
    info->upsampfac = p->sigma;
    info->n_unique = p->n_u;
    info->n_bl = p->n_bl;
    info->n_src = p->n_src;
    for (int i = 0; i < 3; ++i) {
        info->nf1_max[i] = p->nf1_max[i];
        info->nf2_max[i] = p->M_max[i];
        info->src_centre[i] = p->C[i];
        info->src_halfwidth[i] = p->S[i];
    }
    info->workspace_bytes = p->ws_bytes;
    info->transform = p->use_basis ? FV_TRANSFORM_BASIS : (p->use_lattice ? FV_TRANSFORM_LATTICE : FV_TRANSFORM_TYPE3);
    info->basis_terms = p->use_basis ? p->n_basis : 0;
    info->basis_fit_error = p->use_basis && p->n_basis_req == 0 ? p->basis_fit_err : -1.0;
    info->height_terms = p->use_lattice || p->use_basis ? 0 : p->hK;
    info->spread_method = p->spread_method;
    for (int i = 0; i < 3; ++i) info->basis_grid[i] = p->use_basis ? p->bg.dim[i].nf1 : 0;
    info->lattice = p->lat_ok ? 1 : 0;
    for (int k = 0; k < 2; ++k) {
        info->lattice_modes[k] = p->use_lattice ? 2 * p->lat_H[k] + 1 : 0;
        info->lattice_grid[k] = p->use_lattice ? p->lg.nf[k] : 0;
    }
    info->lattice_terms = p->use_lattice ? p->lg.K : 0;
    for (int k = 0; k < 4; ++k) info->lattice_basis[k] = p->lat_basis[k];
    info->beam_groups = (int)p->groups.size();
    return FV_OK;
}

fv_status fv_profile_enable(fv_plan_t p, int enable)
{
    if (!p) return FV_ERR_ARG;
    if (cudaSetDevice(p->device) != cudaSuccess) return p->fail(FV_ERR_CUDA, "cudaSetDevice failed");
    if (!enable) CK(prof_harvest(p));
    p->prof_on = enable != 0;
    return FV_OK;
}

fv_status fv_profile_read(fv_plan_t p, fv_profile_data *out)
{
    if (!p || !out) return FV_ERR_ARG;
    if (cudaSetDevice(p->device) != cudaSuccess) return p->fail(FV_ERR_CUDA, "cudaSetDevice failed");
    CK(prof_harvest(p));
    for (int c = 0; c < FV_PROFILE_CLASSES; ++c) {
        out->name[c] = k_prof_names[c];
        out->total_ms[c] = p->prof_ms[c];
        out->launches[c] = p->prof_launches[c];
        out->bytes[c] = p->prof_bytes[c];
        p->prof_ms[c] = 0.0;
        p->prof_launches[c] = 0;
        p->prof_bytes[c] = 0.0;
    }
    return FV_OK;
}

}  // extern "C"
