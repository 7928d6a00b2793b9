// DCA finding and RSS (Algorithm 2, Eq. 1, Sec. 2.2.2).
//
// Layout of the work: a CTA of 128 threads owns 128/LPS seeds; LPS lanes share a seed and split its
// wires (LPS = 1 for large seed counts, 4 when there are too few seeds to fill the GPU).  The wire
// geometry, the CSR hit offsets and (when they fit) the drift distances and masks are staged in
// shared memory with the bulk-copy engine (cp.async.bulk + mbarrier), in tiles of 256 wires.
//
// Closest recorded state of a (seed, wire) pair, found exactly without visiting every state: the
// recorded states of a seed are cut into segments of G consecutive states, at most N1MAX segments.
// A state within G/2 recording intervals of a segment's centre is within R1 = (G/2) h_rec of it in
// space (consecutive recorded states are at most h_rec apart along the track), so
//     dist(any state of segment j) >= dist(centre j) - R1.
// The centres live in shared memory.  Segments whose bound exceeds the best centre distance cannot
// hold the closest state; they are skipped.  The remaining segments (the union over the warp, so the
// loads stay coalesced: all lanes read the same state index of 32 consecutive seeds) are scanned in
// full, keeping the lexicographic minimum (distance, index).  Scanning a superset of the segments that
// can hold the minimum returns the same minimum.
//
// Without dca_out, a wire whose closest recorded state is farther than (largest unmasked drift +
// lambda + h_rec/2) is not refined: the true DCA is then at least (largest drift + lambda), so every
// residual |D - r| of that wire is at least lambda and the wire adds exactly lambda^2 to the RSS.
// The same bound also drops segments beyond that distance from the candidate set.
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

template <typename T>
struct Cfg;
template <>
struct Cfg<float> {
    static constexpr int N1MAX = 32;
};
template <>
struct Cfg<double> {
    static constexpr int N1MAX = 16;
};

constexpr size_t align16(size_t x) { return (x + 15) & ~size_t(15); }

template <typename T, int LPS>
struct Smem {
    static constexpr int SPB = kThreads / LPS;
    static constexpr size_t bar = 0;
    static constexpr size_t c1 = 16;
    static constexpr size_t wrow = align16(c1 + sizeof(T) * Cfg<T>::N1MAX * 3 * SPB);
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
    constexpr int N1MAX = Cfg<T>::N1MAX;
    extern __shared__ __align__(128) unsigned char sm[];
    uint64_t *bar = (uint64_t *)(sm + L::bar);
    T *c1 = (T *)(sm + L::c1);
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
    const T R1 = (T)a.R1;
    const T half_rec = (T)a.half_rec;
    const T h_rec = (T)a.h_rec;
    const int G = a.G;

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
    const int n1 = (nv + G - 1) / G;
    for (int j = sub; j < N1MAX; j += LPS) {
        T x = T(0), y = T(0), z = T(0);
        if (valid && j < n1) {
            const int k = min(j * G + G / 2, nv - 1);
            const int64_t o = (int64_t)k * S + s;
            x = P[o];
            y = P[plane + o];
            z = P[2 * plane + o];
        }
        c1[(j * 3 + 0) * SPB + ls] = x;
        c1[(j * 3 + 1) * SPB + ls] = y;
        c1[(j * 3 + 2) * SPB + ls] = z;
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

            // level 1: segment centres from shared memory
            T bd = T(INFINITY);
            int bk = 0x7fffffff;
            T d2a[N1MAX];
#pragma unroll
            for (int j = 0; j < N1MAX; ++j) {
                T d2 = T(INFINITY);
                if (want && j < n1) {
                    d2 = line_dist2<T>(c1[(j * 3 + 0) * SPB + ls], c1[(j * 3 + 1) * SPB + ls],
                                       c1[(j * 3 + 2) * SPB + ls], ax, ay, az, ux, uy, uz);
                    lex_min<T>(bd, bk, d2, min(j * G + G / 2, nv - 1));
                }
                d2a[j] = d2;
            }
            uint32_t cand = 0;
            if (want) {
                T thr = sqrt(bd);
                if (!a.exact_all) thr = fmin(thr, cap + half_rec);
                const T lim = thr + R1;
                const T lim2 = lim * lim;
#pragma unroll
                for (int j = 0; j < N1MAX; ++j)
                    if (d2a[j] <= lim2) cand |= 1u << j;
            }
            uint32_t ucand = __reduce_or_sync(0xffffffffu, cand);

            // level 2: every state of the candidate segments (warp-uniform order)
            while (ucand) {
                const int j = __ffs(ucand) - 1;
                ucand &= ucand - 1;
                const int k0 = j * G;
                for (int t = 0; t < G; ++t) {
                    const int k = k0 + t;
                    if (want && k < nv) {
                        const int64_t o = (int64_t)k * S + s;
                        const T d2 = line_dist2<T>(P[o], P[plane + o], P[2 * plane + o], ax, ay, az,
                                                   ux, uy, uz);
                        lex_min<T>(bd, bk, d2, k);
                    }
                }
            }

            // refinement from the closest recorded state (skipped when the wire cannot contribute)
            const bool refine = want && (a.exact_all || sqrt(bd) <= cap + half_rec);
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

int dca_n1max(comet_dtype dt) { return dt == COMET_F32 ? Cfg<float>::N1MAX : Cfg<double>::N1MAX; }

cudaError_t launch_dca(comet_dtype dt, const comet_field &f, const DcaArgs &a, cudaStream_t st)
{
    return dt == COMET_F32 ? dca_dispatch<float>(f, a, st) : dca_dispatch<double>(f, a, st);
}

} // namespace comet
