// Hand-written mixed-radix (2, 3, 4, 5) FFT pass for the oversampled grid
// (Section 2.2, step 2: "Oversampled FFT").
//
// One pass transforms every row of its input along the row's contiguous axis:
//   load the N grid values of the row, multiply by the deconvolution prescale
//   1/Phihat(l w pi / M) (Section 2.2, step 3a, applied on the grid side of the
//   inner transform), place them at l - N/2 (mod M) in a zero-padded length-M
//   vector, run a Stockham autosort FFT with the sign e^{+2 pi i l m / M}, and
//   keep only the band m in [-H, B-1-H] that the interpolation reads, written
//   transposed as out[b][row].
// The transposed write rotates the axes so that the next pass again reads
// contiguous rows; after d passes the band grid is [b_z][b_y][b_x][pol].
#include "fv_internal.cuh"

namespace fv {

size_t fft_pass_smem_bytes(int M, int elem_bytes) { return (size_t)2 * M * 2 * elem_bytes; }

int fft_max_M(int elem_bytes)
{
    // two ping-pong buffers of M complex values within 227 KB of shared memory
    return (int)(232448 / (4 * elem_bytes));
}

// R-point DFT with the + sign on v[0..R-1] (in place).
template <class G>
__device__ __forceinline__ void dft_small(cpx<G> *v, int R)
{
    if (R == 2) {
        cpx<G> a = v[0], b = v[1];
        v[0] = cadd(a, b);
        v[1] = csub(a, b);
    } else if (R == 4) {
        cpx<G> s02 = cadd(v[0], v[2]), d02 = csub(v[0], v[2]);
        cpx<G> s13 = cadd(v[1], v[3]), d13 = cmuli(csub(v[1], v[3]));
        v[0] = cadd(s02, s13);
        v[2] = csub(s02, s13);
        v[1] = cadd(d02, d13);
        v[3] = csub(d02, d13);
    } else if (R == 3) {
        const G h = (G)0.86602540378443864676;   // sin(2 pi / 3)
        cpx<G> t = cadd(v[1], v[2]), u = cmuli(cscale(csub(v[1], v[2]), h));
        cpx<G> m = csub(v[0], cscale(t, (G)0.5));
        v[0] = cadd(v[0], t);
        v[1] = cadd(m, u);
        v[2] = csub(m, u);
    } else if (R == 5) {
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
}

template <class G>
__global__ void __launch_bounds__(256) k_fft_pass(const cpx<G> *__restrict__ in, cpx<G> *__restrict__ out, long rows,
                                                  DimGeom dg, const G *__restrict__ pre,
                                                  const cpx<G> *__restrict__ tw)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cpx<G> *buf0 = reinterpret_cast<cpx<G> *>(smem_raw);
    cpx<G> *buf1 = buf0 + dg.M;
    const int M = dg.M, N = dg.nf1, B = dg.B, H = dg.H;
    const int tid = threadIdx.x, nt = blockDim.x;
    for (long r = blockIdx.x; r < rows; r += gridDim.x) {
        for (int i = tid; i < M; i += nt) buf0[i] = cmk<G>((G)0, (G)0);
        __syncthreads();
        const cpx<G> *src = in + (size_t)r * N;
        for (int l = tid; l < N; l += nt) {
            int m = l - N / 2;
            if (m < 0) m += M;
            buf0[m] = cscale(src[l], pre[l]);
        }
        __syncthreads();
        cpx<G> *x = buf0, *y = buf1;
        int Ns = 1;
        for (int s = 0; s < dg.nstages; ++s) {
            const int R = dg.radix[s];
            const int MR = M / R;
            const int twstep = M / (Ns * R);
            for (int j = tid; j < MR; j += nt) {
                const int k = j % Ns;
                cpx<G> v[5];
                for (int q = 0; q < R; ++q) v[q] = x[j + q * MR];
                if (Ns > 1)
                    for (int q = 1; q < R; ++q) v[q] = cmul(v[q], tw[q * k * twstep]);
                dft_small(v, R);
                const int base = (j / Ns) * Ns * R + k;
                for (int q = 0; q < R; ++q) y[base + q * Ns] = v[q];
            }
            __syncthreads();
            cpx<G> *t = x; x = y; y = t;
            Ns *= R;
        }
        for (int b = tid; b < B; b += nt) {
            int m = (b - H) % M;
            if (m < 0) m += M;
            out[(size_t)b * rows + r] = x[m];
        }
        __syncthreads();
    }
}

template <class G>
cudaError_t launch_fft_pass(const cpx<G> *in, cpx<G> *out, long rows, const DimGeom &dg, const G *pre,
                            const cpx<G> *tw, cudaStream_t st)
{
    if (rows <= 0) return cudaSuccess;
    size_t smem = fft_pass_smem_bytes(dg.M, sizeof(G));
    // the dynamic shared-memory limit is a per-device function attribute
    static bool attr_set[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (!attr_set[dev]) {
        e = cudaFuncSetAttribute(k_fft_pass<G>, cudaFuncAttributeMaxDynamicSharedMemorySize, 232448);
        if (e != cudaSuccess) return e;
        attr_set[dev] = true;
    }
    unsigned grid = (unsigned)(rows < 1048576 ? rows : 1048576);
    k_fft_pass<G><<<grid, 256, smem, st>>>(in, out, rows, dg, pre, tw);
    return cudaGetLastError();
}

template cudaError_t launch_fft_pass<double>(const cpx<double> *, cpx<double> *, long, const DimGeom &,
                                             const double *, const cpx<double> *, cudaStream_t);
template cudaError_t launch_fft_pass<float>(const cpx<float> *, cpx<float> *, long, const DimGeom &, const float *,
                                            const cpx<float> *, cudaStream_t);

}  // namespace fv
