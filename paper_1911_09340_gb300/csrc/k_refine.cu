// Reference seeds of an iterative scan (Sec. 2.1): the seeds of lowest RSS become reference points
// for a finer scan in their vicinity, kept sparse enough that the new seed sets do not overlap.
//
// refine_refs_kernel (one warp): walks the candidates idx[0..M) in their given order (ascending RSS,
// as comet_scan_select returns them) and accepts a candidate unless, for some accepted reference,
// every lattice coordinate (z0, phi, pz, pT) differs by less than twice the new half-width: the two
// new lattices (reference +- half-width) would then overlap.  Lane j holds accepted reference j, so
// each candidate costs one lane-parallel test and one vote.  phi differences are taken modulo 2 pi.
#include <math.h>

#include "device.cuh"
#include "internal.h"

namespace comet {

namespace {

template <typename T>
__global__ void __launch_bounds__(32) refine_refs_kernel(RefArgs a)
{
    const int lane = threadIdx.x;
    const T *__restrict__ sd = (const T *)a.seeds;
    const int64_t S = a.S;
    double mine[4] = {0.0, 0.0, 0.0, 0.0};   // accepted reference `lane`
    int n = 0;
    for (int c = 0; c < a.M && n < a.K; ++c) {
        const int64_t s = a.idx[c];
        if (s < 0 || s >= S) continue;   // unused slot of a short selection
        const double px = (double)sd[3 * S + s], py = (double)sd[4 * S + s];
        const double v[4] = {(double)sd[2 * S + s], atan2(py, px), (double)sd[5 * S + s], hypot(px, py)};
        bool overlap = lane < n;
#pragma unroll
        for (int d = 0; d < 4; ++d) {
            double dv = v[d] - mine[d];
            if (d == 1) dv = remainder(dv, 6.283185307179586);   // 2 pi
            overlap = overlap && fabs(dv) < 2.0 * a.half_width[d];
        }
        if (__any_sync(0xffffffffu, overlap)) continue;
        if (lane == n) {
#pragma unroll
            for (int d = 0; d < 4; ++d) mine[d] = v[d];
        }
        ++n;
    }
    if (lane < n) {
#pragma unroll
        for (int d = 0; d < 4; ++d) a.refs_out[lane * 4 + d] = mine[d];
    }
    if (lane == 0) *a.n_refs_out = n;
}

} // namespace

cudaError_t launch_refine_refs(comet_dtype dt, const RefArgs &a, cudaStream_t st)
{
    if (dt == COMET_F32)
        refine_refs_kernel<float><<<1, 32, 0, st>>>(a);
    else
        refine_refs_kernel<double><<<1, 32, 0, st>>>(a);
    return cudaGetLastError();
}

} // namespace comet
