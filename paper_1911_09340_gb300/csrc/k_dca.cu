// DCA finding and RSS (Algorithm 2, Eq. 1, Sec. 2.2.2).
//
// Layout of the work: a CTA of 128 threads owns 128/LPS seeds; LPS lanes share a seed and split its
// wires (LPS = 1 for large seed counts, 4 when there are too few seeds to fill the GPU).  The wire
// geometry, the CSR hit offsets and (when they fit) the drift distances and masks are staged in
// shared memory with the bulk-copy engine (cp.async.bulk + mbarrier), in tiles of 256 wires.
//
// Closest recorded state of a (seed, wire) pair, found exactly without visiting every state: the
// recorded states of a seed are cut into at most N0MAX super-segments of G0 states, each cut into
// level-1 segments of G1 states.  A state within g/2 recording intervals of a segment's centre is
// within R = (g/2) h_rec of it in space (consecutive recorded states are at most h_rec apart along
// the track), so dist(any state of the segment) >= dist(centre) - R.  The super-segment centres of
// each seed live in shared memory; the level-1 centres and the states are read from the track array.
// At each level a segment is visited only if its bound does not exceed the best distance found so
// far; visiting a superset of the segments that can hold the minimum returns the same lexicographic
// (distance, index) minimum.  Candidate sets are united over the warp so that every load is
// warp-uniform in the state index (32 consecutive seeds: one 128-byte line); the seed lattice numbers
// neighbouring nodes consecutively, so the 32 tracks of a warp are close and the union stays small.
//
// Without dca_out, a wire whose closest recorded state is farther than (largest unmasked drift +
// lambda + h_rec/2) is not refined: the true DCA is then at least (largest drift + lambda), so every
// residual |D - r| of that wire is at least lambda and the wire adds exactly lambda^2 to the RSS.
// The same bound drops segments at every level (a segment is skipped only if it cannot hold a state
// within that distance, or if it cannot hold the minimum).
//
// RSS: each lane sums its wires' d_i^2 in ascending wire order (FP32 as a TwoSum pair, FP64 plainly);
// lanes sharing a seed are combined in a fixed shuffle tree.  No atomics: the result does not depend
// on scheduling (the paper's GPU kernel used atomics and was not deterministic, Sec. 4.1).
#include <float.h>

#include "device.cuh"
#include "internal.h"

namespace comet {

namespace {

constexpr int kThreads = 128;
constexpr int kWireTile = 256;
constexpr int kWireCap = kWireTile + 32;     // elements per staged row (room for the 16-B shift)
constexpr int kHitMax = 1024;                // hits staged in shared memory when H <= kHitMax
constexpr int kHitCap = kHitMax + 32;
constexpr uint64_t kWaitNs = 2000000000ull;  // bulk-copy wait limit (2 s)

// super-segment centres per seed kept in shared memory; level-1 segments per super-segment
constexpr int kN0Max = 16;
constexpr int kN1Max = 32;

constexpr size_t align16(size_t x) { return (x + 15) & ~size_t(15); }

template <typename T, int LPS>
struct Smem {
    static constexpr int SPB = kThreads / LPS;
    static constexpr size_t bar = 0;
    static constexpr size_t c0 = 16;
    static constexpr size_t wrow = align16(c0 + sizeof(T) * kN0Max * 3 * SPB);
    static constexpr size_t orow = align16(wrow + sizeof(T) * 6 * kWireCap);
    static constexpr size_t cap = align16(orow + sizeof(int32_t) * (kWireCap + 8));
    static constexpr size_t drift = align16(cap + sizeof(T) * kWireTile);
    static constexpr size_t mask = align16(drift + sizeof(T) * kHitCap);
    static constexpr size_t total = align16(mask + kHitCap);
};

// Plans the staging of one array, issues its bulk copy (thread 0) and plain-loads its ragged ends
// (all threads).  Returns the element offset of element 0 in dst.
template <typename E>
__device__ __forceinline__ int stage_issue(E *dst, const E *src, int n, uint64_t *bar, bool issuer)
{
    const StagePlan p = stage_plan(src, n, (int)sizeof(E));
    if (issuer && p.body > 0)
        bulk_g2s(dst + p.off + p.head, src + p.head, (uint32_t)(p.body * sizeof(E)), bar);
    for (int i = threadIdx.x; i < p.head; i += blockDim.x) dst[p.off + i] = src[i];
    for (int i = p.head + p.body + threadIdx.x; i < n; i += blockDim.x) dst[p.off + i] = src[i];
    return p.off;
}

template <typename E>
__device__ __forceinline__ uint32_t stage_bytes(const E *src, int n)
{
    const StagePlan p = stage_plan(src, n, (int)sizeof(E));
    return (uint32_t)(p.body * sizeof(E));
}

// After a timed-out wait: copy the bulk parts with plain loads.
template <typename E>
__device__ __forceinline__ void stage_fallback(E *dst, const E *src, int n)
{
    const StagePlan p = stage_plan(src, n, (int)sizeof(E));
    for (int i = p.head + threadIdx.x; i < p.head + p.body; i += blockDim.x) dst[p.off + i] = src[i];
}

// Twosum accumulator for FP32, plain for FP64.
template <typename T>
struct Acc;
template <>
struct Acc<float> {
    float hi = 0.f, lo = 0.f;
    __device__ __forceinline__ void add(float v) { two_sum_add(hi, lo, v); }
    __device__ __forceinline__ void add_pair(float h2, float l2)
    {
        two_sum_add(hi, lo, h2);
        two_sum_add(hi, lo, l2);
    }
    __device__ __forceinline__ float value() const { return hi + lo; }
};
template <>
struct Acc<double> {
    double hi = 0.0, lo = 0.0;
    __device__ __forceinline__ void add(double v) { hi += v; }
    __device__ __forceinline__ void add_pair(double h2, double) { hi += h2; }
    __device__ __forceinline__ double value() const { return hi; }
};

} // namespace

template <typename T, class F, int LPS>
__global__ void __launch_bounds__(kThreads) dca_kernel(F f, DcaArgs a)
{
    using L = Smem<T, LPS>;
    constexpr int SPB = L::SPB;
    extern __shared__ __align__(128) unsigned char sm[];
    uint64_t *bar = (uint64_t *)(sm + L::bar);
    T *c0 = (T *)(sm + L::c0);
    T *wrow = (T *)(sm + L::wrow);
    int32_t *orow = (int32_t *)(sm + L::orow);
    T *capv = (T *)(sm + L::cap);
    T *dsm = (T *)(sm + L::drift);
    uint8_t *msm = (uint8_t *)(sm + L::mask);

    const int tid = threadIdx.x;
    const int ls = tid / LPS;
    const int sub = tid % LPS;
    const int64_t S = a.S;
    const int64_t s = (int64_t)blockIdx.x * SPB + ls;
    const bool valid = s < S;
    const T *__restrict__ P = (const T *)a.points;
    const int64_t plane = (int64_t)a.n_rec * S;
    const T *__restrict__ Wg = (const T *)a.wires;
    const T *__restrict__ Dg = (const T *)a.drift;
    const T lam = (T)a.lambda;
    const T tol = (T)a.tol;
    const T R0 = (T)a.R0;
    const T R1 = (T)a.R1;
    const T half_rec = (T)a.half_rec;
    const T h_rec = (T)a.h_rec;
    const int G0 = a.G0, G1 = a.G1;
    const int N1 = (G0 + G1 - 1) / G1;

    if (tid == 0) mbar_init(bar, 1);

    // per-seed constants and the level-1 centres
    int nv = 1;
    T c = T(0), ip = T(0);
    if (valid) {
        nv = a.n_valid[s];
        const int q = a.charge[s];
        const double px = P[3 * plane + s], py = P[4 * plane + s], pz = P[5 * plane + s];
        const double pd = sqrt(px * px + py * py + pz * pz);
        c = (T)(kKappa * q / pd);
        ip = (T)(1.0 / pd);
    }
    const int n0 = (nv + G0 - 1) / G0;
    for (int j = sub; j < kN0Max; j += LPS) {
        T x = T(0), y = T(0), z = T(0);
        if (valid && j < n0) {
            const int k = min(j * G0 + G0 / 2, nv - 1);
            const int64_t o = (int64_t)k * S + s;
            x = P[o];
            y = P[plane + o];
            z = P[2 * plane + o];
        }
        c0[(j * 3 + 0) * SPB + ls] = x;
        c0[(j * 3 + 1) * SPB + ls] = y;
        c0[(j * 3 + 2) * SPB + ls] = z;
    }

    const int W = a.W;
    const int H = W > 0 ? a.offs[W] : 0;
    const bool hits_sm = H <= kHitMax;
    uint32_t parity = 0;
    bool any_timeout = false;
    int doff = 0, moff = 0;
    __syncthreads();   // barrier initialised, centres written

    // hits: staged once per CTA when they fit
    if (hits_sm && H > 0) {
        const uint32_t bytes = stage_bytes<T>(Dg, H) + stage_bytes<uint8_t>(a.mask, H);
        if (tid == 0 && bytes > 0) {
            fence_proxy_async_smem();
            mbar_arrive_expect_tx(bar, bytes);
        }
        doff = stage_issue<T>(dsm, Dg, H, bar, tid == 0);
        moff = stage_issue<uint8_t>(msm, a.mask, H, bar, tid == 0);
        bool to = false;
        if (bytes > 0) {
            to = !mbar_wait(bar, parity, kWaitNs);
            parity ^= 1u;
        }
        if (__syncthreads_or(to)) {
            any_timeout = true;
            stage_fallback<T>(dsm, Dg, H);
            stage_fallback<uint8_t>(msm, a.mask, H);
        }
        __syncthreads();
    }

    Acc<T> acc;
    int nin = 0, nunc = 0;

    for (int w0 = 0; w0 < W; w0 += kWireTile) {
        const int wn = min(kWireTile, W - w0);
        // ---- stage the wire tile
        uint32_t bytes = stage_bytes<int32_t>(a.offs + w0, wn + 1);
#pragma unroll
        for (int r = 0; r < 6; ++r) bytes += stage_bytes<T>(Wg + (size_t)r * a.ldw + w0, wn);
        if (tid == 0 && bytes > 0) {
            fence_proxy_async_smem();
            mbar_arrive_expect_tx(bar, bytes);
        }
        int woff[6];
#pragma unroll
        for (int r = 0; r < 6; ++r)
            woff[r] = stage_issue<T>(wrow + r * kWireCap, Wg + (size_t)r * a.ldw + w0, wn, bar, tid == 0);
        const int ooff = stage_issue<int32_t>(orow, a.offs + w0, wn + 1, bar, tid == 0);
        bool to = false;
        if (bytes > 0) {
            to = !mbar_wait(bar, parity, kWaitNs);
            parity ^= 1u;
        }
        if (__syncthreads_or(to)) {
            any_timeout = true;
#pragma unroll
            for (int r = 0; r < 6; ++r)
                stage_fallback<T>(wrow + r * kWireCap, Wg + (size_t)r * a.ldw + w0, wn);
            stage_fallback<int32_t>(orow, a.offs + w0, wn + 1);
        }
        __syncthreads();
        // ---- per-wire capture radius: largest unmasked drift + lambda (-1: no unmasked hit)
        for (int i = tid; i < wn; i += kThreads) {
            const int hb = orow[ooff + i], he = orow[ooff + i + 1];
            T mr = T(-1);
            for (int j = hb; j < he; ++j) {
                const bool m = hits_sm ? msm[moff + j] != 0 : a.mask[j] != 0;
                const T r = hits_sm ? dsm[doff + j] : Dg[j];
                if (!m && r > mr) mr = r;
            }
            capv[i] = mr >= T(0) ? mr + lam : T(-1);
        }
        __syncthreads();

        const T *wax = wrow + 0 * kWireCap + woff[0];
        const T *way = wrow + 1 * kWireCap + woff[1];
        const T *waz = wrow + 2 * kWireCap + woff[2];
        const T *wux = wrow + 3 * kWireCap + woff[3];
        const T *wuy = wrow + 4 * kWireCap + woff[4];
        const T *wuz = wrow + 5 * kWireCap + woff[5];

        // ---- the wires of this tile (trip count uniform across the warp)
        for (int base = 0; base < wn; base += LPS) {
            const int ii = base + sub;
            const bool inw = ii < wn;
            T cap = T(-1), ax = T(0), ay = T(0), az = T(0), ux = T(0), uy = T(0), uz = T(1);
            if (inw) {
                cap = capv[ii];
                ax = wax[ii];
                ay = way[ii];
                az = waz[ii];
                ux = wux[ii];
                uy = wuy[ii];
                uz = wuz[ii];
            }
            const bool want = valid && inw && (cap >= T(0) || a.exact_all);

            // level 0: super-segment centres from shared memory
            T bd = T(INFINITY);
            int bk = 0x7fffffff;
            T d0[kN0Max];
#pragma unroll
            for (int j = 0; j < kN0Max; ++j) {
                T d2 = T(INFINITY);
                if (want && j < n0) {
                    d2 = line_dist2<T>(c0[(j * 3 + 0) * SPB + ls], c0[(j * 3 + 1) * SPB + ls],
                                       c0[(j * 3 + 2) * SPB + ls], ax, ay, az, ux, uy, uz);
                    lex_min<T>(bd, bk, d2, min(j * G0 + G0 / 2, nv - 1));
                }
                d0[j] = d2;
            }
            const T capth = a.exact_all ? T(INFINITY) : cap + half_rec;
            uint32_t cand0 = 0;
            if (want) {
                const T lim = fmin(sqrt(bd), capth) + R0;
                const T lim2 = lim * lim;
#pragma unroll
                for (int j = 0; j < kN0Max; ++j)
                    if (d0[j] <= lim2) cand0 |= 1u << j;
            }
            uint32_t u0 = __reduce_or_sync(0xffffffffu, cand0);

            constexpr int kUnroll = 4;
            while (u0) {
                const int j = __ffs(u0) - 1;
                u0 &= u0 - 1;
                const int sb = j * G0;
                const int se = min(sb + G0, nv);          // this lane's end of super-segment j
                // level 1: centres of the level-1 segments of super-segment j
                uint32_t cand1 = 0;
                {
                    const T lim = want ? fmin(sqrt(bd), capth) + R1 : T(0);
                    const T lim2 = lim * lim;
                    for (int m0 = 0; m0 < N1; m0 += kUnroll) {
                        T xs[kUnroll], ys[kUnroll], zs[kUnroll];
                        int ks[kUnroll];
#pragma unroll
                        for (int u = 0; u < kUnroll; ++u) {
                            const int m = m0 + u;
                            const int st = sb + m * G1;
                            xs[u] = ys[u] = zs[u] = T(0);
                            ks[u] = -1;
                            if (want && m < N1 && st < se) {
                                const int k = min(st + G1 / 2, min(st + G1, se) - 1);
                                const int64_t o = (int64_t)k * S + s;
                                xs[u] = P[o];
                                ys[u] = P[plane + o];
                                zs[u] = P[2 * plane + o];
                                ks[u] = k;
                            }
                        }
#pragma unroll
                        for (int u = 0; u < kUnroll; ++u) {
                            if (ks[u] >= 0) {
                                const T d2 = line_dist2<T>(xs[u], ys[u], zs[u], ax, ay, az, ux, uy, uz);
                                lex_min<T>(bd, bk, d2, ks[u]);
                                if (d2 <= lim2) cand1 |= 1u << (m0 + u);
                            }
                        }
                    }
                }
                uint32_t u1 = __reduce_or_sync(0xffffffffu, cand1);
                // level 2: every state of the candidate level-1 segments
                while (u1) {
                    const int m = __ffs(u1) - 1;
                    u1 &= u1 - 1;
                    const int k0 = sb + m * G1;
                    const int kend = min(k0 + G1, se);
                    for (int t0 = k0; t0 < k0 + G1; t0 += kUnroll) {
                        T xs[kUnroll], ys[kUnroll], zs[kUnroll];
#pragma unroll
                        for (int u = 0; u < kUnroll; ++u) {
                            const int k = t0 + u;
                            xs[u] = ys[u] = zs[u] = T(0);
                            if (want && k < kend) {
                                const int64_t o = (int64_t)k * S + s;
                                xs[u] = P[o];
                                ys[u] = P[plane + o];
                                zs[u] = P[2 * plane + o];
                            }
                        }
#pragma unroll
                        for (int u = 0; u < kUnroll; ++u) {
                            const int k = t0 + u;
                            if (want && k < kend)
                                lex_min<T>(bd, bk, line_dist2<T>(xs[u], ys[u], zs[u], ax, ay, az, ux, uy, uz), k);
                        }
                    }
                }
            }

            // refinement from the closest recorded state (skipped when the wire cannot contribute)
            const bool refine = want && (a.exact_all || sqrt(bd) <= capth);
            T D = T(INFINITY);
            if (refine) {
                T yv[6];
                const int64_t o = (int64_t)bk * S + s;
#pragma unroll
                for (int cc = 0; cc < 6; ++cc) yv[cc] = P[cc * plane + o];
                const int conv = refine_dca<T, F>(f, c, ip, yv, ax, ay, az, ux, uy, uz, tol,
                                                  a.max_iter, h_rec, D);
                if (cap >= T(0)) nunc += 1 - conv;
                if (a.dca_out) ((T *)a.dca_out)[(int64_t)(w0 + ii) * S + s] = D;
            }
            if (valid && inw && cap >= T(0)) {
                T emin = T(INFINITY);
                if (refine) {
                    const int hb = orow[ooff + ii], he = orow[ooff + ii + 1];
                    for (int j = hb; j < he; ++j) {
                        const bool m = hits_sm ? msm[moff + j] != 0 : a.mask[j] != 0;
                        if (m) continue;
                        const T r = hits_sm ? dsm[doff + j] : Dg[j];
                        const T e = fabs(D - r);
                        emin = e < emin ? e : emin;
                    }
                }
                const T d = emin < lam ? emin : lam;
                nin += emin < lam ? 1 : 0;
                acc.add(d * d);
            }
        }
        __syncthreads();   // tile consumed before the next staging overwrites it
    }

    // combine the lanes of a seed in a fixed order
#pragma unroll
    for (int off = LPS / 2; off > 0; off >>= 1) {
        const T oh = __shfl_xor_sync(0xffffffffu, acc.hi, off);
        const T ol = __shfl_xor_sync(0xffffffffu, acc.lo, off);
        const int on = __shfl_xor_sync(0xffffffffu, nin, off);
        if ((sub & off) == 0) {
            acc.add_pair(oh, ol);
            nin += on;
        }
    }
    if (valid && sub == 0) {
        ((T *)a.rss)[s] = acc.value();
        a.n_in[s] = nin;
    }
    if (a.n_unconv) {
        int t = nunc;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) t += __shfl_xor_sync(0xffffffffu, t, off);
        if ((tid & 31) == 0 && t) atomicAdd(a.n_unconv, t);
    }
    if (any_timeout) {
        if (tid == 0 && a.status) atomicOr(a.status, 1);
        // no bulk copy may still be writing into shared memory when the CTA exits
        mbar_wait(bar, parity ^ 1u, kWaitNs);
    }
}

template <typename T, class F, int LPS>
static cudaError_t dca_launch_one(const F &fld, const DcaArgs &a, cudaStream_t st)
{
    using L = Smem<T, LPS>;
    static const cudaError_t attr = cudaFuncSetAttribute(
        dca_kernel<T, F, LPS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L::total);
    if (attr != cudaSuccess) return attr;
    const int64_t nb = (a.S + L::SPB - 1) / L::SPB;
    dca_kernel<T, F, LPS><<<(unsigned)nb, kThreads, L::total, st>>>(fld, a);
    return cudaGetLastError();
}

template <typename T, class F>
static cudaError_t dca_lps(const F &fld, const DcaArgs &a, cudaStream_t st)
{
    // fewer seeds than ~8 resident threads per FP32 lane of the GPU: share seeds among 4 lanes
    if (a.S < 65536) return dca_launch_one<T, F, 4>(fld, a, st);
    return dca_launch_one<T, F, 1>(fld, a, st);
}

template <typename T>
static cudaError_t dca_dispatch(const comet_field &f, const DcaArgs &a, cudaStream_t st)
{
    switch (field_kind(f)) {
    case FieldKind::Axial:
        return dca_lps<T>(FieldAxial<T>{(T)f.b[2]}, a, st);
    case FieldKind::Uniform:
        return dca_lps<T>(FieldUniform<T>{(T)f.b[0], (T)f.b[1], (T)f.b[2]}, a, st);
    case FieldKind::Table:
    default:
        return dca_lps<T>(FieldTable<T>{(const float *)f.table, f.nx, f.ny, f.nz, (T)f.origin[0],
                                        (T)f.origin[1], (T)f.origin[2], (T)(1.0 / f.spacing)},
                          a, st);
    }
}

void dca_segments(int n_rec, int *G0, int *G1)
{
    // about cbrt(n_rec) super-segments of about sqrt(G0)-state level-1 segments
    int n0 = (int)lround(cbrt((double)n_rec));
    n0 = n0 < 2 ? 2 : (n0 > kN0Max ? kN0Max : n0);
    int g0 = (n_rec + n0 - 1) / n0;
    if ((n_rec + g0 - 1) / g0 > kN0Max) g0 = (n_rec + kN0Max - 1) / kN0Max;
    int g1 = (int)lround(sqrt((double)g0));
    g1 = g1 < 1 ? 1 : g1;
    if ((g0 + g1 - 1) / g1 > kN1Max) g1 = (g0 + kN1Max - 1) / kN1Max;
    *G0 = g0;
    *G1 = g1;
}

cudaError_t launch_dca(comet_dtype dt, const comet_field &f, const DcaArgs &a, cudaStream_t st)
{
    return dt == COMET_F32 ? dca_dispatch<float>(f, a, st) : dca_dispatch<double>(f, a, st);
}

} // namespace comet
