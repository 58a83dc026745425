// Staged source records for the gather spreading (Section 2.2, step 1): the
// record layout that the prep kernel writes and the spreading kernel copies into
// shared memory in bulk, and the launchers of both.
#pragma once
#include "fv_internal.cuh"

namespace fv {

// Status bits a kernel may set in the plan's device status word.
#define FV_DEVICE_TIMEOUT 1

// One source of one slice as the gather spreader reads it (16- or 32-byte records, copied in bulk):
// cell = cx | cy << 14 | cz << 28 (first footprint cell per axis; cx, cy < 16384, cz < 16) and the
// offsets frac = l0 - q of the grid coordinate split (Section 2.2).
template <class G> struct SrcRec;
template <> struct __align__(16) SrcRec<float> {
    unsigned cell;
    float fx, fy, fz;
};
template <> struct __align__(16) SrcRec<double> {
    unsigned cell, pad;
    double fx, fy, fz;
};

// Complex strengths per source in the staged layout: n_pol values padded to a multiple of 16 bytes.
__host__ __device__ inline int staged_cs_stride(int elem, int n_pol)   // complex elements per source
{
    const int bytes = n_pol * 2 * elem;
    return ((bytes + 15) & ~15) / (2 * elem);
}

// The gather spreading (launch_spread_tile) reading staged records: each CTA's candidate chunks are copied
// into shared memory in bulk, double buffered.  Writes every cell of grid [n_pol][nz][ny][nx].
// status: device word; FV_DEVICE_TIMEOUT is or-ed in if a bounded wait on a copy ran out (the grid is
// then zero).  rec and cs must be readable 16 bytes past the last visible source.
template <class G>
cudaError_t launch_spread_gather_rec(const int *offsets, const SrcRec<G> *rec, const cpx<G> *cs, const SliceGeom &g,
                                     const TimeBin &tb, double r0, double r1, int *status, cpx<G> *grid,
                                     cudaStream_t st);

// Per slice: strengths with prephase and packed grid coordinates of the sorted sources, as staged
// records (the same arithmetic as launch_prep).
template <class G>
cudaError_t launch_prep_staged(const double *sdir, const int *sidx, const int *nv_ptr, long n_src,
                               const void *flux, int flux_fp64, int n_freq, int f, const SliceGeom &g,
                               SrcRec<G> *rec, cpx<G> *cs, cudaStream_t st);

// FP32 grids: the same, from the per-time records tc of launch_time_binning (no FP64 arithmetic); writes
// staged records when rec is given, else cell[3][n] / frac[3][n] / cs[n_pol][n].
cudaError_t launch_prep_tc(const float4 *tc, const int *sidx, const int *nv_ptr, long n_src, const void *flux,
                           int flux_fp64, int n_freq, int f, const SliceGeom &g, int *cell, float *frac,
                           cpx<float> *cs, SrcRec<float> *rec, cudaStream_t st);

}  // namespace fv
