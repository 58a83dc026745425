// Hand-written mixed-radix (2, 3, 4, 5, 8) FFT pass for the oversampled grid
// (Section 2.2, step 2: "Oversampled FFT").
//
// One pass transforms every row of its input along the row's contiguous axis:
//   load the N grid values of the row, multiply by the deconvolution prescale
//   1/Phihat(l w pi / M) of this axis (Section 2.2, step 3a, applied on the
//   grid side of the inner transform), place them at l - N/2 (mod M) of a
//   zero-padded length-M vector, run a Stockham autosort FFT with the sign
//   e^{+2 pi i l m / M}, and keep only the band m in [-H, B-1-H] that the
//   interpolation reads, written transposed as out[b][row].
// The transposed write rotates the axes so that the next pass again reads
// contiguous rows.
//
// GB300 mapping: a CTA holds R consecutive rows in shared memory (R chosen so
// that R*M <= kSmemElems), so the transposed store writes R consecutive
// complex values per band index, and neighbouring CTAs fill the rest of each
// 32-byte sector.  Stockham stages ping-pong between two shared buffers; a
// thread keeps one radix-RD butterfly (compile-time radix) in registers.
#include "fv_internal.cuh"

namespace fv {

static constexpr int kThreads = 256;

template <class G> struct FftCfg;
template <> struct FftCfg<float> { static constexpr int kSmemElems = 4096; };    // 2 x 32 KB of complex64
template <> struct FftCfg<double> { static constexpr int kSmemElems = 2048; };   // 2 x 32 KB of complex128

size_t fft_pass_smem_bytes(int M, int elem_bytes)
{
    const int cap = elem_bytes == 4 ? FftCfg<float>::kSmemElems : FftCfg<double>::kSmemElems;
    int R = cap / M;
    if (R < 1) R = 1;
    if (R > 8) R = 8;
    return (size_t)2 * R * M * 2 * elem_bytes;
}

// longest row: two buffers of one row within 192 KB of shared memory
int fft_max_M(int elem_bytes) { return elem_bytes == 4 ? 12288 : 6144; }

static int rows_per_cta(int M, int elem_bytes)
{
    const int cap = elem_bytes == 4 ? FftCfg<float>::kSmemElems : FftCfg<double>::kSmemElems;
    int R = cap / M;
    return R < 1 ? 1 : (R > 8 ? 8 : R);
}

// R-point DFT with the + sign, in registers.
template <class G, int R> struct Dft;
template <class G> struct Dft<G, 2> {
    static __device__ __forceinline__ void run(cpx<G> *v)
    {
        cpx<G> a = v[0], b = v[1];
        v[0] = cadd(a, b);
        v[1] = csub(a, b);
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
template <class G> struct Dft<G, 8> {
    // radix 8 = radix 2 over two radix-4 halves with the e^{+2 pi i k/8} twiddles
    static __device__ __forceinline__ void run(cpx<G> *v)
    {
        const G r = (G)0.70710678118654752440;
        cpx<G> e[4] = {v[0], v[2], v[4], v[6]}, o[4] = {v[1], v[3], v[5], v[7]};
        Dft<G, 4>::run(e);
        Dft<G, 4>::run(o);
        // o[k] *= e^{+2 pi i k / 8}
        o[1] = cmk<G>(r * (o[1].x - o[1].y), r * (o[1].x + o[1].y));
        o[2] = cmuli(o[2]);
        o[3] = cmk<G>(-r * (o[3].x + o[3].y), r * (o[3].x - o[3].y));
        for (int k = 0; k < 4; ++k) {
            v[k] = cadd(e[k], o[k]);
            v[k + 4] = csub(e[k], o[k]);
        }
    }
};

// One Stockham stage of radix RD over the R rows: x -> y.
template <class G, int RD>
__device__ __forceinline__ void stage(const cpx<G> *__restrict__ x, cpx<G> *__restrict__ y, int M, int R, int Ns,
                                      const cpx<G> *__restrict__ tw)
{
    const int MR = M / RD;
    const int per = R * MR;
    const int twstep = M / (Ns * RD);
    for (int bi = threadIdx.x; bi < per; bi += kThreads) {
        const int row = bi / MR;
        const int j = bi - row * MR;
        const int k = j % Ns;
        const cpx<G> *src = x + row * M + j;
        cpx<G> v[RD];
#pragma unroll
        for (int q = 0; q < RD; ++q) v[q] = src[q * MR];
        if (Ns > 1) {
#pragma unroll
            for (int q = 1; q < RD; ++q) v[q] = cmul(v[q], tw[q * k * twstep]);
        }
        Dft<G, RD>::run(v);
        cpx<G> *dst = y + row * M + (j / Ns) * Ns * RD + k;
#pragma unroll
        for (int q = 0; q < RD; ++q) dst[q * Ns] = v[q];
    }
    __syncthreads();
}

template <class G>
__global__ void __launch_bounds__(kThreads) k_fft_rows(const cpx<G> *__restrict__ in, cpx<G> *__restrict__ out,
                                                       long rows, DimGeom dg, const G *__restrict__ pre,
                                                       const cpx<G> *__restrict__ tw, int R)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cpx<G> *sm = reinterpret_cast<cpx<G> *>(smem_raw);
    const int M = dg.M, N = dg.nf1, B = dg.B, H = dg.H;
    const int half = N / 2;
    for (long row0 = (long)blockIdx.x * R; row0 < rows; row0 += (long)gridDim.x * R) {
        const int nr = (int)((rows - row0) < R ? (rows - row0) : R);
        // load + prescale + zero padding: slot m holds l = m + N/2 (m < N - N/2) or l = m - M + N/2
        for (int idx = threadIdx.x; idx < R * M; idx += kThreads) {
            const int r = idx / M;
            const int m = idx - r * M;
            int l = -1;
            if (m < N - half) l = m + half;
            else if (m >= M - half) l = m - M + half;
            cpx<G> v = cmk<G>((G)0, (G)0);
            if (l >= 0 && r < nr) v = cscale(in[(size_t)(row0 + r) * N + l], pre[l]);
            sm[idx] = v;
        }
        __syncthreads();
        cpx<G> *x = sm, *y = sm + R * M;
        int Ns = 1;
        for (int s = 0; s < dg.nstages; ++s) {
            const int rd = dg.radix[s];
            if (rd == 8) stage<G, 8>(x, y, M, R, Ns, tw);
            else if (rd == 4) stage<G, 4>(x, y, M, R, Ns, tw);
            else if (rd == 2) stage<G, 2>(x, y, M, R, Ns, tw);
            else if (rd == 3) stage<G, 3>(x, y, M, R, Ns, tw);
            else stage<G, 5>(x, y, M, R, Ns, tw);
            cpx<G> *t = x; x = y; y = t;
            Ns *= rd;
        }
        // band output, transposed: consecutive threads write consecutive rows of one band index
        for (int idx = threadIdx.x; idx < B * nr; idx += kThreads) {
            const int b = idx / nr;
            const int r = idx - b * nr;
            int m = (b - H) % M;
            if (m < 0) m += M;
            out[(size_t)b * rows + row0 + r] = x[r * M + m];
        }
        __syncthreads();
    }
}

template <class G>
cudaError_t launch_fft_pass(const cpx<G> *in, cpx<G> *out, long rows, const DimGeom &dg, const G *pre,
                            const cpx<G> *tw, cudaStream_t st)
{
    if (rows <= 0) return cudaSuccess;
    if (dg.M > fft_max_M(sizeof(G))) return cudaErrorInvalidValue;
    const int R = rows_per_cta(dg.M, sizeof(G));
    const size_t smem = (size_t)2 * R * dg.M * sizeof(cpx<G>);
    static bool attr_set[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (!attr_set[dev]) {
        e = cudaFuncSetAttribute(k_fft_rows<G>, cudaFuncAttributeMaxDynamicSharedMemorySize, 196608);
        if (e != cudaSuccess) return e;
        attr_set[dev] = true;
    }
    long ctas = (rows + R - 1) / R;
    unsigned grid = (unsigned)(ctas < 1048576 ? ctas : 1048576);
    k_fft_rows<G><<<grid, kThreads, smem, st>>>(in, out, rows, dg, pre, tw, R);
    return cudaGetLastError();
}

template cudaError_t launch_fft_pass<double>(const cpx<double> *, cpx<double> *, long, const DimGeom &,
                                             const double *, const cpx<double> *, cudaStream_t);
template cudaError_t launch_fft_pass<float>(const cpx<float> *, cpx<float> *, long, const DimGeom &, const float *,
                                            const cpx<float> *, cudaStream_t);

}  // namespace fv
