// Hand-written mixed-radix FFT pass for the oversampled grid (Section 2.2,
// step 2: "Oversampled FFT").
//
// One pass transforms every row of its input along the row's contiguous axis:
//   load the N grid values of the row, multiply by the deconvolution prescale
//   1/Phihat(l w pi / M) of this axis (Section 2.2, step 3a, applied on the
//   grid side of the inner transform; pre = nullptr when the spreading kernel
//   already applied it), place them at l - N/2 (mod M) of a
//   zero-padded length-M vector, run a Stockham autosort FFT with the sign
//   e^{+2 pi i l m / M}, and keep only the band m in [-H, B-1-H] that the
//   interpolation reads, written transposed as out[b][row].
// The transposed write rotates the axes so that the next pass again reads
// contiguous rows.
//
// GB300 mapping.  M is chosen as a product of at most three (four beyond
// 4096) radices from {2,3,4,5,6,8,9,10,12,15,16}, so a row takes at most
// three trips through shared memory; each radix-R butterfly runs in
// registers (composite R as nested Cooley-Tukey with compile-time twiddles).
// A CTA holds R_rows consecutive rows in two padded shared buffers (one
// complex of padding per 16, which breaks the bank conflicts of the
// stride-R stores of the first stage); index arithmetic uses
// multiply-high division by the per-stage constants prepared on the host.
#include "fv_internal.cuh"

namespace fv {

static constexpr int kThreads = 256;

// ---------------------------------------------------------------- compile-time twiddles
// e^{2 pi i m / R} for 2 <= R <= 16, from Taylor series on [0, pi/4] after an
// exact reduction of the rational angle m/R to an octant (constexpr, host compiler).
namespace cx {
constexpr double kPi = 3.14159265358979323846264338327950288;
constexpr double sin_t(double a)
{
    double t = a, s = a;
    for (int n = 1; n < 12; ++n) {
        t *= -a * a / ((2.0 * n) * (2.0 * n + 1.0));
        s += t;
    }
    return s;
}
constexpr double cos_t(double a)
{
    double t = 1.0, s = 1.0;
    for (int n = 1; n < 12; ++n) {
        t *= -a * a / ((2.0 * n - 1.0) * (2.0 * n));
        s += t;
    }
    return s;
}
struct SC { double s, c; };
constexpr SC sincos2pi(int m, int R)
{
    m %= R;
    if (m < 0) m += R;
    const long t = 4L * m;
    const int k = (int)(t / R);            // quarter turns
    const long rem = t - (long)k * R;      // remaining angle (pi/2) rem / R
    double s0 = 0, c0 = 0;
    if (2 * rem <= R) {
        const double a = (kPi / 2) * (double)rem / R;
        s0 = sin_t(a);
        c0 = cos_t(a);
    } else {
        const double a = (kPi / 2) * (double)(R - rem) / R;
        s0 = cos_t(a);
        c0 = sin_t(a);
    }
    if (k == 0) return {s0, c0};
    if (k == 1) return {c0, -s0};
    if (k == 2) return {-s0, -c0};
    return {-c0, s0};
}
}  // namespace cx

// v * e^{2 pi i m / R} with compile-time m, R: exact for the quarter turns, otherwise a product by
// constants folded at compile time (no table load, no FP64 conversion in the FP32 instances)
template <class G, int M_, int R>
__device__ __forceinline__ cpx<G> twm(cpx<G> v)
{
    constexpr int m = M_ % R;
    if constexpr (m == 0) return v;
    else if constexpr (4 * m == R) return cmuli(v);
    else if constexpr (2 * m == R) return cmk<G>(-v.x, -v.y);
    else if constexpr (4 * m == 3 * R) return cmk<G>(v.y, -v.x);
    else {
        constexpr cx::SC w = cx::sincos2pi(m, R);
        return cmul(v, cmk<G>((G)w.c, (G)w.s));
    }
}

// ---------------------------------------------------------------- register DFTs (+ sign)
template <int R> struct Fac {
    static constexpr int A = (R % 4 == 0 && R != 4) ? 4 : (R % 2 == 0 && R != 2) ? 2 : (R % 3 == 0 && R != 3) ? 3 : 5;
    static constexpr int B = R / A;
};

template <class G, int R> struct Dft;

template <class G> struct Dft<G, 2> {
    static __device__ __forceinline__ void run(cpx<G> *v)
    {
        cpx<G> a = v[0], b = v[1];
        v[0] = cadd(a, b);
        v[1] = csub(a, b);
    }
};
template <class G> struct Dft<G, 3> {
    static __device__ __forceinline__ void run(cpx<G> *v)
    {
        const G h = (G)0.86602540378443864676;   // sin(2 pi / 3)
        cpx<G> t = cadd(v[1], v[2]), u = cmuli(cscale(csub(v[1], v[2]), h));
        cpx<G> m = csub(v[0], cscale(t, (G)0.5));
        v[0] = cadd(v[0], t);
        v[1] = cadd(m, u);
        v[2] = csub(m, u);
    }
};
template <class G> struct Dft<G, 4> {
    static __device__ __forceinline__ void run(cpx<G> *v)
    {
        cpx<G> s02 = cadd(v[0], v[2]), d02 = csub(v[0], v[2]);
        cpx<G> s13 = cadd(v[1], v[3]), d13 = cmuli(csub(v[1], v[3]));
        v[0] = cadd(s02, s13);
        v[2] = csub(s02, s13);
        v[1] = cadd(d02, d13);
        v[3] = csub(d02, d13);
    }
};
template <class G> struct Dft<G, 5> {
    static __device__ __forceinline__ void run(cpx<G> *v)
    {
        const G c1 = (G)0.30901699437494742410, c2 = (G)-0.80901699437494742410;   // cos(2pi/5), cos(4pi/5)
        const G s1 = (G)0.95105651629515357212, s2 = (G)0.58778525229247312917;    // sin(2pi/5), sin(4pi/5)
        cpx<G> t1 = cadd(v[1], v[4]), t2 = cadd(v[2], v[3]);
        cpx<G> u1 = csub(v[1], v[4]), u2 = csub(v[2], v[3]);
        cpx<G> a1 = cadd(v[0], cadd(cscale(t1, c1), cscale(t2, c2)));
        cpx<G> a2 = cadd(v[0], cadd(cscale(t1, c2), cscale(t2, c1)));
        cpx<G> b1 = cmuli(cadd(cscale(u1, s1), cscale(u2, s2)));
        cpx<G> b2 = cmuli(csub(cscale(u1, s2), cscale(u2, s1)));
        v[0] = cadd(v[0], cadd(t1, t2));
        v[1] = cadd(a1, b1);
        v[4] = csub(a1, b1);
        v[2] = cadd(a2, b2);
        v[3] = csub(a2, b2);
    }
};

// Composite R = A B: with r = B r1 + r2 and q = q1 + A q2,
// w_R^{rq} = w_A^{r1 q1} w_R^{r2 q1} w_B^{r2 q2}:
// A-point DFTs over r1 for every r2, twiddles w_R^{r2 q1}, B-point DFTs over r2.
template <class G, int R, int A, int R2, int Q1>
__device__ __forceinline__ void col_twiddle(const cpx<G> *t, cpx<G> *u)
{
    if constexpr (Q1 < A) {
        u[Q1] = twm<G, R2 * Q1, R>(t[Q1]);
        col_twiddle<G, R, A, R2, Q1 + 1>(t, u);
    }
}

template <class G, int R, int A, int B, int R2>
__device__ __forceinline__ void col_pass(const cpx<G> *v, cpx<G> (*U)[A])
{
    if constexpr (R2 < B) {
        cpx<G> t[A];
#pragma unroll
        for (int r1 = 0; r1 < A; ++r1) t[r1] = v[B * r1 + R2];
        Dft<G, A>::run(t);
        col_twiddle<G, R, A, R2, 0>(t, U[R2]);
        col_pass<G, R, A, B, R2 + 1>(v, U);
    }
}

template <class G, int R> struct Dft {
    static __device__ __forceinline__ void run(cpx<G> *v)
    {
        constexpr int A = Fac<R>::A, B = Fac<R>::B;
        cpx<G> U[B][A];
        col_pass<G, R, A, B, 0>(v, U);
#pragma unroll
        for (int q1 = 0; q1 < A; ++q1) {
            cpx<G> t[B];
#pragma unroll
            for (int r2 = 0; r2 < B; ++r2) t[r2] = U[r2][q1];
            Dft<G, B>::run(t);
#pragma unroll
            for (int q2 = 0; q2 < B; ++q2) v[q1 + A * q2] = t[q2];
        }
    }
};

// ---------------------------------------------------------------- stages
__device__ __forceinline__ unsigned fdiv(unsigned n, unsigned mul, unsigned sh)
{
    return (__umulhi(n, mul) + n) >> sh;
}
__device__ __forceinline__ int pad(int i) { return i + (i >> 4); }

// Where a stage's input and output live.  The first stage reads the
// zero-padded row without the padding ever being stored: positions in
// [zlo, zhi) are zeros.  The last stage (Ns = M / RD, so j = k and its
// outputs are the frequencies m = k + q Ns) writes only the band, straight to
// global memory, transposed: out[b][row] with b = m + H (mod M), every b < B.
template <class G> struct StageIO {
    int zlo, zhi;                 // first stage: zero positions of the input row
    cpx<G> *out;                  // last stage: band output (nullptr: write y)
    long rows, row0;
    int nr, B, H;
    float inv_nrows;
};

template <class G, int RD>
__device__ __forceinline__ void stage(const cpx<G> *__restrict__ x, cpx<G> *__restrict__ y, const DimGeom &dg,
                                      int s, int nrows, int Ns, const cpx<G> *__restrict__ tw, bool first,
                                      StageIO<G> io)
{
    const int M = dg.M;
    const int MR = M / RD;
    const int per = nrows * MR;
    const int twstep = M / (Ns * RD);
    const bool last = io.out != nullptr;
    for (int bi = threadIdx.x; bi < per; bi += kThreads) {
        int row, j;
        if (last) {
            // row fastest, so that consecutive threads write consecutive rows of one band index
            j = (int)(((float)bi + 0.5f) * io.inv_nrows);
            row = bi - j * nrows;
        } else {
            row = (int)fdiv((unsigned)bi, dg.mr_mul[s], dg.mr_sh[s]);
            j = bi - row * MR;
        }
        const int jq = last ? 0 : (int)fdiv((unsigned)j, dg.ns_mul[s], dg.ns_sh[s]);
        const int k = j - jq * Ns;
        const int base = row * M;
        cpx<G> v[RD];
        if (first) {
#pragma unroll
            for (int q = 0; q < RD; ++q) {
                const int pos = j + q * MR;
                v[q] = (pos >= io.zlo && pos < io.zhi) ? cmk<G>((G)0, (G)0) : x[pad(base + pos)];
            }
        } else {
#pragma unroll
            for (int q = 0; q < RD; ++q) v[q] = x[pad(base + j + q * MR)];
        }
        if (Ns > 1) {
            if constexpr (sizeof(G) == 4) {
                // FP32: twiddles w^q, w = e^{2 pi i k / (Ns RD)}, from one table load and RD - 2 products
                // (the FMA pipe has room, the load pipe less; the products add a few ulps, measured
                // 9.2e-7 -> 9.4e-7 of relative L2 on the mixed 127-antenna workload)
                const cpx<G> w1 = tw[k * twstep];
                cpx<G> wq = w1;
#pragma unroll
                for (int q = 1; q < RD; ++q) {
                    v[q] = cmul(v[q], wq);
                    if (q + 1 < RD) wq = cmul(wq, w1);
                }
            } else {
                // FP64: products would run on the narrow FP64 pipe, so every twiddle comes from the table
#pragma unroll
                for (int q = 1; q < RD; ++q) v[q] = cmul(v[q], tw[q * k * twstep]);
            }
        }
        Dft<G, RD>::run(v);
        if (last) {
            if (row < io.nr) {
#pragma unroll
                for (int q = 0; q < RD; ++q) {
                    int b = k + q * Ns + io.H;
                    while (b >= M) b -= M;
                    for (; b < io.B; b += M) io.out[(size_t)b * io.rows + io.row0 + row] = v[q];
                }
            }
        } else {
            const int o = base + jq * Ns * RD + k;
#pragma unroll
            for (int q = 0; q < RD; ++q) y[pad(o + q * Ns)] = v[q];
        }
    }
    __syncthreads();
}

template <class G, int MAXRD>
__device__ __forceinline__ void run_stage(int rd, const cpx<G> *x, cpx<G> *y, const DimGeom &dg, int s, int nrows,
                                          int Ns, const cpx<G> *tw, bool first, StageIO<G> io)
{
    switch (rd) {
    case 2: stage<G, 2>(x, y, dg, s, nrows, Ns, tw, first, io); break;
    case 3: stage<G, 3>(x, y, dg, s, nrows, Ns, tw, first, io); break;
    case 4: stage<G, 4>(x, y, dg, s, nrows, Ns, tw, first, io); break;
    case 5: stage<G, 5>(x, y, dg, s, nrows, Ns, tw, first, io); break;
    case 6: stage<G, 6>(x, y, dg, s, nrows, Ns, tw, first, io); break;
    case 8: stage<G, 8>(x, y, dg, s, nrows, Ns, tw, first, io); break;
    default:
        if constexpr (MAXRD > 8) {
            switch (rd) {
            case 9: stage<G, 9>(x, y, dg, s, nrows, Ns, tw, first, io); break;
            case 10: stage<G, 10>(x, y, dg, s, nrows, Ns, tw, first, io); break;
            case 12: stage<G, 12>(x, y, dg, s, nrows, Ns, tw, first, io); break;
            case 15: stage<G, 15>(x, y, dg, s, nrows, Ns, tw, first, io); break;
            default: stage<G, 16>(x, y, dg, s, nrows, Ns, tw, first, io); break;
            }
        }
        break;
    }
}

// kRowsElems: the input values of one row block held in registers (prefetch); kSmemElems: the
// transform points of one row block in shared memory (rows per CTA = kSmemElems / M).  FP32: 6,144
// points, i.e. two rows of 3,072 (measured 16 % faster x passes than one row per CTA: three butterflies
// per thread and stage instead of one or two), the prefetch covering their 2 x 1,500 inputs.
template <class G> struct FftCfg;
template <> struct FftCfg<float> { static constexpr int kRowsElems = 4096, kSmemElems = 6144; };
template <> struct FftCfg<double> { static constexpr int kRowsElems = 2048, kSmemElems = 2048; };

int fft_rows_per_cta(int M, int elem_bytes)
{
    const int cap = elem_bytes == 4 ? FftCfg<float>::kSmemElems : FftCfg<double>::kSmemElems;
    int R = cap / M;
    return R < 1 ? 1 : (R > 8 ? 8 : R);
}

__host__ __device__ __forceinline__ size_t buf_elems(int R, int M) { return (size_t)R * M + ((size_t)R * M >> 4) + 1; }

size_t fft_pass_smem_bytes(int M, int elem_bytes)
{
    return 2 * buf_elems(fft_rows_per_cta(M, elem_bytes), M) * 2 * elem_bytes;
}

// longest row: two padded buffers of one row within 200 KB of shared memory
int fft_max_M(int elem_bytes) { return elem_bytes == 4 ? 12000 : 6000; }

// Input of one row block, held in registers between blocks so that the
// global loads of block i+1 are in flight while block i runs its stages.
template <class G> struct Prefetch {
    static constexpr int kMax = FftCfg<G>::kRowsElems / kThreads;   // values per thread
    cpx<G> v[kMax];
};

template <class G>
__device__ __forceinline__ void prefetch_rows(Prefetch<G> &pf, const cpx<G> *__restrict__ in, long rows, long row0,
                                              int R, int N)
{
    const int tot = R * N;
#pragma unroll
    for (int k = 0; k < Prefetch<G>::kMax; ++k) {
        const int idx = threadIdx.x + k * kThreads;
        const long r = row0 + idx / N;
        pf.v[k] = (idx < tot && r < rows) ? in[row0 * N + idx] : cmk<G>((G)0, (G)0);
    }
}

// resident CTAs per SM the register allocation must allow (FP32 radix <= 8: 3 CTAs at <= 80 registers
// without spills; the wider instances need more registers per thread)
template <class G, int MAXRD> struct FftMinBlocks {
    static constexpr int value = sizeof(G) == 4 ? (MAXRD <= 8 ? 3 : 2) : 1;
};

template <class G, int MAXRD>
__global__ void __launch_bounds__(kThreads, (FftMinBlocks<G, MAXRD>::value)) k_fft_rows(const cpx<G> *__restrict__ in, cpx<G> *__restrict__ out,
                                                       long rows, DimGeom dg, const G *__restrict__ pre,
                                                       const cpx<G> *__restrict__ tw, int R)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int M = dg.M, N = dg.nf1, B = dg.B, H = dg.H;
    cpx<G> *buf0 = reinterpret_cast<cpx<G> *>(smem_raw);
    cpx<G> *buf1 = buf0 + buf_elems(R, M);
    const int half = N / 2;
    const long stride = (long)gridDim.x * R;
    Prefetch<G> pf;
    long row0 = (long)blockIdx.x * R;
    if (row0 < rows) prefetch_rows(pf, in, rows, row0, R, N);
    for (; row0 < rows; row0 += stride) {
        const int nr = (int)((rows - row0) < R ? (rows - row0) : R);
        // the prefetched row values with the prescale: l -> slot (l - N/2) mod M; the other slots are
        // zeros that are never stored (the first stage knows where they are)
#pragma unroll
        for (int k = 0; k < Prefetch<G>::kMax; ++k) {
            const int idx = threadIdx.x + k * kThreads;
            if (idx < R * N) {
                const int r = idx / N;
                const int l = idx - r * N;
                int m = l - half;
                if (m < 0) m += M;
                buf0[pad(r * M + m)] = pre ? cscale(pf.v[k], pre[l]) : pf.v[k];
            }
        }
        // a row longer than the prefetch holds (then R = 1): the rest of it straight from memory
        for (int idx = Prefetch<G>::kMax * kThreads + threadIdx.x; idx < R * N; idx += kThreads) {
            const int r = idx / N;
            const int l = idx - r * N;
            int m = l - half;
            if (m < 0) m += M;
            const cpx<G> v = row0 + r < rows ? in[row0 * N + idx] : cmk<G>((G)0, (G)0);
            buf0[pad(r * M + m)] = pre ? cscale(v, pre[l]) : v;
        }
        __syncthreads();
        // issue the next block's loads before the stages
        if (row0 + stride < rows) prefetch_rows(pf, in, rows, row0 + stride, R, N);
        cpx<G> *x = buf0, *y = buf1;
        int Ns = 1;
        StageIO<G> io{N - half, M - half, nullptr, rows, row0, nr, B, H, 1.0f / (float)R};
        for (int s = 0; s < dg.nstages; ++s) {
            const int rd = dg.radix[s];
            io.out = s == dg.nstages - 1 ? out : nullptr;
            run_stage<G, MAXRD>(rd, x, y, dg, s, R, Ns, tw, s == 0, io);
            cpx<G> *t = x; x = y; y = t;
            Ns *= rd;
        }
    }
}

template <class G, int MAXRD>
static cudaError_t launch_rows(const cpx<G> *in, cpx<G> *out, long rows, const DimGeom &dg, const G *pre,
                               const cpx<G> *tw, cudaStream_t st)
{
    const int R = fft_rows_per_cta(dg.M, sizeof(G));
    const size_t smem = 2 * buf_elems(R, dg.M) * sizeof(cpx<G>);
    static bool attr_set[64] = {};
    static int max_ctas[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (!attr_set[dev]) {
        e = cudaFuncSetAttribute(k_fft_rows<G, MAXRD>, cudaFuncAttributeMaxDynamicSharedMemorySize, 210000);
        if (e != cudaSuccess) return e;
        attr_set[dev] = true;
    }
    // persistent CTAs: as many as fit on the device for the largest configuration (each keeps a
    // row block of prefetch in registers)
    if (!max_ctas[dev]) {
        int sms = 0;
        e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return e;
        max_ctas[dev] = sms;
    }
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fft_rows<G, MAXRD>, kThreads, smem);
    if (e != cudaSuccess) return e;
    const long cap = (long)max_ctas[dev] * (per_sm > 0 ? per_sm : 1);
    const long ctas = (rows + R - 1) / R;
    const unsigned grid = (unsigned)(ctas < cap ? ctas : cap);
    k_fft_rows<G, MAXRD><<<grid, kThreads, smem, st>>>(in, out, rows, dg, pre, tw, R);
    return cudaGetLastError();
}

template <class G>
cudaError_t launch_fft_pass(const cpx<G> *in, cpx<G> *out, long rows, const DimGeom &dg, const G *pre,
                            const cpx<G> *tw, cudaStream_t st)
{
    if (rows <= 0) return cudaSuccess;
    if (dg.M > fft_max_M(sizeof(G)) || dg.nstages < 1) return cudaErrorInvalidValue;
    int maxrd = 1;
    for (int s = 0; s < dg.nstages; ++s) maxrd = dg.radix[s] > maxrd ? dg.radix[s] : maxrd;
    if (maxrd <= 8) return launch_rows<G, 8>(in, out, rows, dg, pre, tw, st);
    return launch_rows<G, 16>(in, out, rows, dg, pre, tw, st);
}

template cudaError_t launch_fft_pass<double>(const cpx<double> *, cpx<double> *, long, const DimGeom &,
                                             const double *, const cpx<double> *, cudaStream_t);
template cudaError_t launch_fft_pass<float>(const cpx<float> *, cpx<float> *, long, const DimGeom &, const float *,
                                            const cpx<float> *, cudaStream_t);

// ---------------------------------------------------------------- host planning
static const int kRadices[] = {16, 15, 12, 10, 9, 8, 6, 5, 4, 3, 2};

static bool factor_into(int M, int maxStages, int maxRadix, int *rad, int &n)
{
    if (M == 1) return true;
    if (maxStages == 0) return false;
    for (int r : kRadices)
        if (r <= maxRadix && M % r == 0) {
            rad[n++] = r;
            if (factor_into(M / r, maxStages - 1, maxRadix, rad, n)) return true;
            --n;
        }
    return false;
}

// multiply-high division by d: q = (umulhi(n, mul) + n) >> sh for n < 2^31
static void magic_u32(unsigned d, unsigned &mul, unsigned &sh)
{
    unsigned s = 0;
    while ((1ull << s) < d) ++s;
    sh = s;
    mul = (unsigned)((((1ull << 32) * ((1ull << s) - d)) / d) + 1);
}

int fft_choose_length(int target, int *radix, int &nstages, int maxRadix)
{
    if (maxRadix < 2) maxRadix = 16;
    // stage budget: enough stages of maxRadix to reach the target, at least 3
    int maxStages = 3;
    for (long span = (long)maxRadix * maxRadix * maxRadix; span < target && maxStages < FV_MAX_STAGES; span *= maxRadix)
        ++maxStages;
    for (int M = target + (target & 1); M <= 4 * target + 64; M += 2) {
        int n = 0;
        if (factor_into(M, maxStages, maxRadix, radix, n)) {
            nstages = n;
            return M;
        }
    }
    return -1;
}

void fft_stage_constants(DimGeom &dg)
{
    int Ns = 1;
    for (int s = 0; s < dg.nstages; ++s) {
        magic_u32((unsigned)(dg.M / dg.radix[s]), dg.mr_mul[s], dg.mr_sh[s]);
        magic_u32((unsigned)Ns, dg.ns_mul[s], dg.ns_sh[s]);
        Ns *= dg.radix[s];
    }
}

}  // namespace fv
