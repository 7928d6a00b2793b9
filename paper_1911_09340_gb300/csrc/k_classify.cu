// Hit classification of the selected seed (Sec. 2.1) and the hit mask of the next turn partition
// (Sec. 3.1: hits classified earlier are excluded from later seed scans).
//
// WPW warps per wire: their lanes split the selected seed's recorded states for an exhaustive
// closest-state search and reduce the lexicographic (distance, index) minimum with warp shuffles
// (then, with WPW > 1, across the warps in shared memory); one lane refines the DCA on the virtual
// plane exactly as comet_scan_dca does (same device functions, same inputs, hence the same D), then
// classifies the closest unmasked hit if |D - r| < lambda.  The minimum does not depend on how the
// states are split, so every WPW gives the same results.  The batched launch packs 8 wires into a
// block (WPW 1); a single-event launch has a few hundred wires at most and gives each its own block
// of 4 warps, so that a partition with few wires still spreads over the SMs.
#include <float.h>

#include "device.cuh"
#include "internal.h"

namespace comet {

// BATCH: one launch for a batch of events; block b belongs to the event that batch_find gives
// (8 wires per block).
template <typename T, class F, bool BATCH, int WPW>
__global__ void __launch_bounds__(256) classify_kernel(F f, ClsArgs a, BatchLaunch L)
{
    int64_t bx = blockIdx.x;
    if constexpr (BATCH) {
        int e;
        int64_t lb;
        if (!batch_find(L.cls_start, L.B, blockIdx.x, e, lb)) return;
        a = L.ev[e].cls;
        bx = lb;
    }
    const int lane = threadIdx.x & 31;
    const int warp = WPW > 1 ? (int)(threadIdx.x >> 5) : 0;
    const int i = WPW > 1 ? (int)bx : (int)((bx * blockDim.x + threadIdx.x) >> 5);
    if (i >= a.W) return;   // whole warps (whole blocks when WPW > 1)
    const int hb = a.offs[i], he = a.offs[i + 1];
    const int64_t s = *a.seed_index;
    if (s < 0 || s >= a.S) {   // the same for every thread of the block
        if (warp == 0) {
            for (int j = hb + lane; j < he; j += 32) a.hit_class[j] = 0;
            if (lane == 0 && a.status) atomicOr(a.status, 2);
        }
        return;
    }
    const int64_t S = a.S;
    const int64_t plane = (int64_t)a.n_rec * S;
    const T *__restrict__ P = (const T *)a.points;
    const T *__restrict__ Wg = (const T *)a.wires;
    const T ax = Wg[i], ay = Wg[(size_t)a.ldw + i], az = Wg[2 * (size_t)a.ldw + i];
    const T ux = Wg[3 * (size_t)a.ldw + i], uy = Wg[4 * (size_t)a.ldw + i],
            uz = Wg[5 * (size_t)a.ldw + i];
    const int nv = a.n_valid[s];

    // same frame and distance as comet_scan_dca's search, so both find the same closest state
    [[maybe_unused]] const WireFrame<T> fr = wire_frame<T>(ax, ay, az, ux, uy, uz);
    T bd = T(INFINITY);
    int bk = 0x7fffffff;
    for (int k = warp * 32 + lane; k < nv; k += 32 * WPW) {
        const int64_t o = (int64_t)k * S + s;
#if COMET_SEARCH_FRAME
        lex_min<T>(bd, bk,
                   frame_dist2<T>(P[o], P[plane + o], P[2 * plane + o], fr.vx, fr.vy, fr.vz, fr.av,
                                  fr.wx, fr.wy, fr.wz, fr.aw),
                   k);
#else
        lex_min<T>(bd, bk, line_dist2<T>(P[o], P[plane + o], P[2 * plane + o], ax, ay, az, ux, uy, uz),
                   k);
#endif
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        const T od = __shfl_xor_sync(0xffffffffu, bd, off);
        const int ok = __shfl_xor_sync(0xffffffffu, bk, off);
        lex_min<T>(bd, bk, od, ok);
    }
    if constexpr (WPW > 1) {
        __shared__ T s_bd[WPW];
        __shared__ int s_bk[WPW];
        if (lane == 0) {
            s_bd[warp] = bd;
            s_bk[warp] = bk;
        }
        __syncthreads();
        if (threadIdx.x != 0) return;
        for (int w = 1; w < WPW; ++w) lex_min<T>(bd, bk, s_bd[w], s_bk[w]);
    } else {
        if (lane != 0) return;
    }

    T c, ip;
    seed_kinematics<T>(P[3 * plane + s], P[4 * plane + s], P[5 * plane + s], a.charge[s], c, ip);
    T y[6];
    const int64_t o = (int64_t)bk * S + s;
#pragma unroll
    for (int c = 0; c < 6; ++c) y[c] = P[c * plane + o];
    T D;
    refine_dca<T, F>(f, c, ip, y, ax, ay, az, ux, uy, uz, (T)a.tol, a.max_iter, (T)a.h_rec, D);
    if (a.dca_wire) ((T *)a.dca_wire)[i] = D;

    const T *__restrict__ Dg = (const T *)a.drift;
    const T lam = (T)a.lambda;
    int jb = -1;
    T eb = T(INFINITY);
    for (int j = hb; j < he; ++j) {
        if (a.mask[j]) continue;
        const T e = fabs(D - Dg[j]);
        if (e < eb) {
            eb = e;
            jb = j;
        }
    }
    for (int j = hb; j < he; ++j) {
        const uint8_t cl = (j == jb && eb < lam) ? 1 : 0;
        a.hit_class[j] = cl;
        if (cl && a.update_mask) a.mask[j] = 1;
    }
}

template <typename T, bool BATCH, int WPW>
static void cls_dispatch(const comet_field &f, const ClsArgs &a, unsigned nb, const BatchLaunch &L,
                         cudaStream_t st)
{
    const int nt = WPW > 1 ? 32 * WPW : 256;
    switch (field_kind(f)) {
    case FieldKind::Axial:
        classify_kernel<T, FieldAxial<T>, BATCH, WPW><<<nb, nt, 0, st>>>(FieldAxial<T>{(T)f.b[2]}, a, L);
        break;
    case FieldKind::Uniform:
        classify_kernel<T, FieldUniform<T>, BATCH, WPW><<<nb, nt, 0, st>>>(
            FieldUniform<T>{(T)f.b[0], (T)f.b[1], (T)f.b[2]}, a, L);
        break;
    case FieldKind::Table:
        classify_kernel<T, FieldTable<T>, BATCH, WPW><<<nb, nt, 0, st>>>(make_table<T>(f), a, L);
        break;
    }
}

cudaError_t launch_classify(comet_dtype dt, const comet_field &f, const ClsArgs &a, cudaStream_t st)
{
    if (a.W == 0) return cudaSuccess;
    const unsigned nb = (unsigned)a.W;   // one block of 4 warps per wire
    if (dt == COMET_F32)
        cls_dispatch<float, false, 4>(f, a, nb, BatchLaunch{}, st);
    else
        cls_dispatch<double, false, 4>(f, a, nb, BatchLaunch{}, st);
    return cudaGetLastError();
}

cudaError_t launch_classify_batch(comet_dtype dt, const comet_field &f, const BatchLaunch &L,
                                  cudaStream_t st)
{
    if (L.cls_blocks == 0) return cudaSuccess;
    if (dt == COMET_F32)
        cls_dispatch<float, true, 1>(f, ClsArgs{}, L.cls_blocks, L, st);
    else
        cls_dispatch<double, true, 1>(f, ClsArgs{}, L.cls_blocks, L, st);
    return cudaGetLastError();
}

} // namespace comet
