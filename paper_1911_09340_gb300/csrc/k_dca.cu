// DCA finding and RSS (Algorithm 2, Eq. 1, Sec. 2.2.2).
//
// Layout of the work: one thread per seed, a warp per 32-seed group.  The persistent kernel (up to
// 1024 wires) stages every wire's geometry, the CSR hit offsets and (when they fit) the drift
// distances and masks once per CTA in shared memory with the bulk-copy engine (cp.async.bulk +
// mbarrier), and its warps take (group, wire chunk) items; the tiled kernel (more wires) stages
// them in tiles of 256 wires per 128-seed CTA.
//
// Closest recorded state of a (seed, wire) pair, found exactly without visiting every state.  The
// recorded states of each seed are cut into at most 8 super-segments of G0 states, each cut into at
// most 24 level-1 segments of G1 states.  Because the seed lattice numbers neighbouring nodes
// consecutively, the 32 tracks of a warp are close, and one bounding sphere per segment covers all
// 32 of them: its centre is the midpoint of the first and the last lane's segment centres, its
// radius the largest distance from it to any lane's segment centre plus (g/2) h_rec (a recorded
// state within g/2 recording intervals of a centre is at most that far from it along the track).
// Every recorded state x of that segment of every seed of the warp then satisfies
// dist(x, wire) >= dist(C, wire) - radius.  The spheres are read in place from the table the
// recording kernel wrote (or built in shared memory when no table is given).  For each wire, the
// lanes test the spheres in parallel (lane t: wire t against the super-segment spheres; then lane
// m: level-1 sphere m of a candidate super-segment) and only segments whose bound does not exceed
// the wire's capture radius (largest unmasked drift + lambda + h_rec/2) are scanned state by
// state, each lane its own seed's states, keeping the lexicographic (distance, index) minimum.  If a seed's closest state is within the capture radius it lies in a
// scanned segment, so the minimum is exact; if not, every residual of the wire is at least lambda
// and the wire adds exactly lambda^2 to the RSS, with or without a refinement.  Beyond the first
// and the last recorded state the refinement reaches up to h_rec (not h_rec/2) from the nearest
// recorded state, so segments that may hold a track end are tested, and an end state refined,
// within capture radius + h_rec.  With dca_out every state is scanned (exact DCA for every wire).
//
// RSS: each thread sums its wires' d_i^2 in ascending wire order within each wire chunk (FP32 as a
// TwoSum pair, FP64 plainly), then the chunks' sums in chunk order.  Atomics only hand out work
// and count arrivals: the result does not depend on scheduling (the paper's GPU kernel summed with
// atomics and was not deterministic, Sec. 4.1).
#include <float.h>

#include "device.cuh"
#include "internal.h"

// Tuning constants (compile-time): minimum resident CTAs per SM requested from the register
// allocator, and how many states are loaded together.
#ifndef COMET_DCA_MINB
#define COMET_DCA_MINB 7
#endif
// FP64: bound by the FP64 pipe rather than by resident warps; fewer CTAs per SM buy registers (at
// 72 the FP64 kernels spill ~300 B per thread)
#ifndef COMET_DCA_MINB_F64
#define COMET_DCA_MINB_F64 4
#endif
// FP32 in a non-axial field (tabulated or general uniform): RK4 stages in the refinement; at 72
// registers the tabulated-field kernel spilled ~200 B per thread
#ifndef COMET_DCA_MINB_FIELD
#define COMET_DCA_MINB_FIELD 5
#endif
#ifndef COMET_DCA_U2
#define COMET_DCA_U2 2
#endif
// 1: the candidate scan loads each state's momentum with its position and keeps the closest
// state, so that the refinement starts without a second dependent load
#ifndef COMET_DCA_SCAN_P
#define COMET_DCA_SCAN_P 1
#endif
// wires per chunk of the per-seed sums (the persistent kernel's finest work item)
#ifndef COMET_DCA_CHUNK_W
#define COMET_DCA_CHUNK_W 32
#endif

namespace comet {

namespace {

constexpr int kThreads = 128;
constexpr int kWarps = kThreads / 32;
static_assert(kWarps == kDcaWarpsPerCta, "persistent DCA CTA size");
constexpr int kWireTile = 256;
constexpr int kWireCap = kWireTile + 32;     // elements per staged row (room for the 16-B shift)
constexpr int kHitMax = 1024;                // hits staged in shared memory when H <= kHitMax
constexpr int kHitCap = kHitMax + 32;
constexpr uint64_t kWaitNs = 2000000000ull;  // limit of the wait for an abandoned copy (2 s)

__host__ __device__ constexpr size_t align16(size_t x) { return (x + 15) & ~size_t(15); }

template <typename T>
struct Smem {
    static constexpr size_t bar = 0;
    static constexpr size_t sph0 = 16;                                            // [warp][j][4]
    static constexpr size_t sph1 = align16(sph0 + sizeof(float) * kWarps * kN0Max * 4);  // [warp][j][m][4]
    static constexpr size_t wrow = align16(sph1 + sizeof(float) * kWarps * kN0Max * kN1Max * 4);
    static constexpr size_t orow = align16(wrow + sizeof(T) * 6 * kWireCap);
    static constexpr size_t cap = align16(orow + sizeof(int32_t) * (kWireCap + 8));
    static constexpr size_t frame = align16(cap + sizeof(T) * kWireTile);
    static constexpr size_t drift = align16(frame + sizeof(T) * 16 * kWireTile);
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

// A launch scalar in the working precision: the host-rounded float copy for FP32.
template <typename T>
__device__ __forceinline__ T in_prec(double d, float f)
{
    if constexpr (sizeof(T) == 4)
        return f;
    else
        return d;
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

// Extra reach (m) when an FP64 kernel tests a sphere in FP32: float rounding of the wire frame (unit
// vectors and the offsets av = a.v, aw = a.w) and of the distance arithmetic moves the distance by
// a few ulp of the coordinates involved, ~1e-7 m per metre of |av| + |aw| + reach; 2 um plus 1 um
// per metre is a generous bound (the FP64 test it stands in for then never rejects more).
__device__ __forceinline__ float sph_margin_f32(double av, double aw)
{
    return 2e-6f + 1e-6f * (float)(fabs(av) + fabs(aw));
}

template <typename T>
__device__ __forceinline__ bool sphere_within(const float4 &sp, T fvx, T fvy, T fvz, T fav, T fwx,
                                              T fwy, T fwz, T faw, T ax, T ay, T az, T ux, T uy,
                                              T uz, T lim)
{
    if (sp.w < 0.f) return false;
#if COMET_SEARCH_FRAME
    const T d2 = frame_dist2<T>((T)sp.x, (T)sp.y, (T)sp.z, fvx, fvy, fvz, fav, fwx, fwy, fwz, faw);
#else
    const T d2 = line_dist2<T>((T)sp.x, (T)sp.y, (T)sp.z, ax, ay, az, ux, uy, uz);
#endif
    const T l = lim + (T)sp.w;
    return d2 <= l * l;
}

// ------------------------------------------------------------------------------------------------
// One 32-seed group (one warp): per-lane seed state, bounding spheres, and the wire loop
// ------------------------------------------------------------------------------------------------

template <typename T>
struct Group {
    int64_t s;       // this lane's seed
    bool valid;
    int nv;          // recorded states of the seed
    int n0w;         // super-segments of the longest track of the warp
    int elo, ehi;    // smallest and largest last state index over the warp's tracks
    T c, ip;         // KAPPA q / P0, 1 / P0
};

template <typename T>
__device__ __forceinline__ Group<T> load_group(const DcaArgs &a, int64_t g, int lane)
{
    const T *__restrict__ P = (const T *)a.points;
    const int64_t S = a.S;
    const int64_t plane = (int64_t)a.n_rec * S;
    Group<T> gr;
    gr.s = g * 32 + lane;
    gr.valid = gr.s < S;
    gr.nv = 1;
    gr.c = T(0);
    gr.ip = T(0);
    if (gr.valid) {
        gr.nv = a.n_valid[gr.s];
        seed_kinematics<T>(P[3 * plane + gr.s], P[4 * plane + gr.s], P[5 * plane + gr.s],
                           a.charge[gr.s], gr.c, gr.ip);
    }
    int n0w = gr.valid ? (gr.nv + a.G0 - 1) / a.G0 : 0;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) n0w = max(n0w, __shfl_xor_sync(0xffffffffu, n0w, off));
    gr.n0w = n0w;
    gr.elo = (int)__reduce_min_sync(0xffffffffu, (unsigned)(gr.valid ? gr.nv - 1 : 0x7fffffff));
    gr.ehi = (int)__reduce_max_sync(0xffffffffu, (unsigned)(gr.valid ? gr.nv - 1 : 0));
    return gr;
}

// The warp's bounding spheres of its super-segments (sph0[j]) and level-1 segments
// (sph1[j * kN1Max + m]), written by lane 0.
template <typename T>
__device__ __forceinline__ void build_spheres(const DcaArgs &a, const Group<T> &gr, int lane,
                                              float4 *sph0, float4 *sph1, int64_t g)
{
    if (g * 32 >= a.S) return;   // no seed in this group: nothing will be searched
    if (a.bounds) {
        // written by comet_scan_propagate: copy this group's table into the warp's slot
        const float4 *src = (const float4 *)a.bounds + g * kBoundsPerGroup;
        for (int i = lane; i < kBoundsPerGroup; i += 32) {
            const float4 v = __ldg(src + i);
            if (i < kN0Max)
                sph0[i] = v;
            else
                sph1[i - kN0Max] = v;
        }
        __syncwarp();
        return;
    }
    const T *__restrict__ P = (const T *)a.points;
    const int64_t S = a.S;
    const int64_t plane = (int64_t)a.n_rec * S;
    const int G0 = a.G0, G1 = a.G1;
    const int N1 = (G0 + G1 - 1) / G1;
    for (int j = 0; j < kN0Max; ++j) {
        const int sb = j * G0, se = min(sb + G0, gr.nv);
        const bool has = gr.valid && sb < gr.nv;
        T x = T(0), y = T(0), z = T(0);
        if (has) {
            const int64_t o = (int64_t)min(sb + G0 / 2, se - 1) * S + gr.s;
            x = P[o];
            y = P[plane + o];
            z = P[2 * plane + o];
        }
        const float4 sp = warp_sphere<T>(has, x, y, z, (T)a.R0);
        if (lane == 0) sph0[j] = sp;
        for (int m = 0; m < N1; ++m) {
            const int st = sb + m * G1;
            const bool h1 = has && st < se;
            T x1 = T(0), y1 = T(0), z1 = T(0);
            if (h1) {
                const int64_t o = (int64_t)min(st + G1 / 2, min(st + G1, se) - 1) * S + gr.s;
                x1 = P[o];
                y1 = P[plane + o];
                z1 = P[2 * plane + o];
            }
            const float4 sp1 = warp_sphere<T>(h1, x1, y1, z1, (T)a.R1);
            if (lane == 0) sph1[j * kN1Max + m] = sp1;
        }
    }
    __syncwarp();
}

// Per-wire record of a staged tile, four of them per wire: (v, a.v), (w, a.w), (a, capture radius),
// (u, 0) -- one 16-byte-aligned load each (two for double).
template <typename T>
struct alignas(16) Q4 {
    T x, y, z, w;
};

// A staged range of wires [w0, w0 + wn) in shared memory.
template <typename T>
struct Tile {
    const T *ax, *ay, *az, *ux, *uy, *uz;   // wire point and direction, element i = wire w0 + i
    const Q4<T> *rec;                        // [wire][4]: (v, a.v), (w, a.w), (a, cap), (u, 0)
    const T *cap;                            // capture radius (< 0: no unmasked hit)
    const int32_t *offs;                     // CSR offsets, element i = wire w0 + i
    const T *dsm;                            // drifts / masks: staged (global hit index) or global
    const uint8_t *msm;
    int w0, wn;
};

// Capture radius and frame of wire i of a staged tile (one thread per wire), packed with its
// point and direction into the wire's four records.
template <typename T>
__device__ __forceinline__ void tile_wire_setup(const Tile<T> &tl, int i, T lam, T *capv, Q4<T> *rec)
{
    const int hb = tl.offs[i], he = tl.offs[i + 1];
    T mr = T(-1);
    for (int j = hb; j < he; ++j)
        if (!tl.msm[j] && tl.dsm[j] > mr) mr = tl.dsm[j];
    const T cap = mr >= T(0) ? mr + lam : T(-1);
    capv[i] = cap;
    const T ax = tl.ax[i], ay = tl.ay[i], az = tl.az[i], ux = tl.ux[i], uy = tl.uy[i], uz = tl.uz[i];
    const WireFrame<T> fr = wire_frame<T>(ax, ay, az, ux, uy, uz);
    rec[4 * i + 0] = Q4<T>{fr.vx, fr.vy, fr.vz, fr.av};
    rec[4 * i + 1] = Q4<T>{fr.wx, fr.wy, fr.wz, fr.aw};
    rec[4 * i + 2] = Q4<T>{ax, ay, az, cap};
    rec[4 * i + 3] = Q4<T>{ux, uy, uz, T(0)};
}

// Wires [wb, we) of one tile for one 32-seed group: accumulates d_i^2, n_in and unconverged counts.
template <typename T, class F>
__device__ __forceinline__ void group_wires(const F &f, const DcaArgs &a, const Group<T> &gr,
                                            const Tile<T> &tl, const float4 *sph0,
                                            const float4 *sph1, int lane, Acc<T> &acc, int &nin,
                                            int &nunc, int wb, int we)
{
    const T *__restrict__ P = (const T *)a.points;
    const int64_t S = a.S;
    const int64_t plane = (int64_t)a.n_rec * S;
    const int64_t s = gr.s;
    const bool valid = gr.valid;
    const int nv = gr.nv;
    const T lam = in_prec<T>(a.lambda, a.lambda_f), tol = in_prec<T>(a.tol, a.tol_f),
            half_rec = in_prec<T>(a.half_rec, a.half_rec_f), h_rec = in_prec<T>(a.h_rec, a.h_rec_f);
    const int G0 = a.G0, G1 = a.G1;
    const int N1 = (G0 + G1 - 1) / G1;
    const Q4<T> *rec = tl.rec;
    constexpr int kU = COMET_DCA_U2;
    // Tighter reach of the refinement from an interior closest state (axial field): at a point of
    // closest approach X* with distance D, the recorded state within delta <= h_rec/2 of it along the
    // track is at most sqrt(D^2 + delta^2) + kappa delta^2 / 2 from the wire (the tangent line from
    // X* moves away from the wire as sqrt(D^2 + delta^2 |t_perp|^2), the track leaves the tangent by
    // at most kappa delta^2 / 2, kappa = |KAPPA q B / P0| its curvature).  So a closest recorded state
    // farther than sqrt(cap^2 + (h_rec/2)^2) + kappa (h_rec/2)^2 / 2 cannot refine to D < cap: the
    // wire adds lambda^2.  kq2 = the warp's largest kappa times (h_rec/2)^2 / 2, plus the margin.
    T kq2 = T(INFINITY);
    if constexpr (F::kAxial) {
        T kap = fabs(gr.c * f.bz);
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) kap = fmax(kap, __shfl_xor_sync(0xffffffffu, kap, off));
        kq2 = T(0.5) * kap * half_rec * half_rec + in_prec<T>(a.margin, a.margin_f);
    }
    const T hq2 = half_rec * half_rec;

    for (int base = wb; base < we; base += 32) {
        const int clen = min(32, we - base);
        // lane t: which super-segments can bring wire base + t within its capture radius
        uint32_t mask0 = 0;
        if (lane < clen) {
            const int iw = base + lane;
            const T capw = tl.cap[iw];
            if (a.exact_all) {
                mask0 = 1u;
            } else if (capw >= T(0)) {
                const T lim = capw + half_rec;
                const Q4<T> r0 = rec[4 * iw + 0], r1 = rec[4 * iw + 1], r2 = rec[4 * iw + 2],
                            r3 = rec[4 * iw + 3];
                if constexpr (sizeof(T) == 8) {
                    // FP64 kernels test the (float) spheres in FP32: the part's FP64 rate is the
                    // limit there.  The reach grows by sph_margin_f32 so that the test stays a
                    // superset of the FP64 one.
                    const float l = (float)lim + sph_margin_f32(r0.w, r1.w);
                    const float v0 = (float)r0.x, v1 = (float)r0.y, v2 = (float)r0.z, va = (float)r0.w;
                    const float w0 = (float)r1.x, w1 = (float)r1.y, w2 = (float)r1.z, wa = (float)r1.w;
                    for (int j = 0; j < gr.n0w; ++j)
                        if (sphere_within<float>(sph0[j], v0, v1, v2, va, w0, w1, w2, wa, (float)r2.x,
                                                 (float)r2.y, (float)r2.z, (float)r3.x, (float)r3.y,
                                                 (float)r3.z, l))
                            mask0 |= 1u << j;
                } else {
                    for (int j = 0; j < gr.n0w; ++j)
                        if (sphere_within<T>(sph0[j], r0.x, r0.y, r0.z, r0.w, r1.x, r1.y, r1.z, r1.w,
                                             r2.x, r2.y, r2.z, r3.x, r3.y, r3.z, lim))
                            mask0 |= 1u << j;
                }
            }
        }
        for (int t = 0; t < clen; ++t) {
            const int ii = base + t;
            const uint32_t m0 = __shfl_sync(0xffffffffu, mask0, t);
            const Q4<T> r2 = rec[4 * ii + 2];
            const T cap = r2.w;
            if (m0 == 0u) {
                // beyond every seed's capture radius (or no unmasked hit): lambda^2 if in the sum
                if (valid && cap >= T(0)) acc.add(lam * lam);
                continue;
            }
            const Q4<T> r0 = rec[4 * ii + 0], r1 = rec[4 * ii + 1], r3 = rec[4 * ii + 3];
            const T ax = r2.x, ay = r2.y, az = r2.z;
            const T ux = r3.x, uy = r3.y, uz = r3.z;
            const T fvx = r0.x, fvy = r0.y, fvz = r0.z, fav = r0.w;
            const T fwx = r1.x, fwy = r1.y, fwz = r1.z, faw = r1.w;
#if COMET_SEARCH_FRAME
            auto sd2 = [&](T x, T y, T z) {
                return frame_dist2<T>(x, y, z, fvx, fvy, fvz, fav, fwx, fwy, fwz, faw);
            };
#else
            auto sd2 = [&](T x, T y, T z) { return line_dist2<T>(x, y, z, ax, ay, az, ux, uy, uz); };
#endif
            const bool want = valid && (cap >= T(0) || a.exact_all);
            const T capth = a.exact_all ? T(INFINITY) : cap + half_rec;
            // interior reach (see kq2): never above capth
            const T thin = a.exact_all ? T(INFINITY) : fmin(capth, sqrt(cap * cap + hq2) + kq2);
            T bd = T(INFINITY);
            int bk = 0x7fffffff;
#if COMET_DCA_SCAN_P
            // the closest state so far, loaded with the scan (no second round trip to refine)
            T by[6] = {T(0), T(0), T(0), T(0), T(0), T(0)};
            // squared distances of the states scanned just before and after the closest one (for
            // the first refinement step) and of the previous state scanned
            T bdm = T(INFINITY), bdp = T(INFINITY), dprev = T(INFINITY);
            int kprev = -2;
#endif
            // scans states [k0, k1) of this lane's seed, kU at a time (span is warp-uniform)
            auto scan = [&](int k0, int k1, int span) {
                // one 64-bit multiply per range; states are S elements apart
                const T *q0 = P + ((int64_t)k0 * S + s);
                for (int t0 = 0; t0 < span; t0 += kU, q0 += kU * S) {
                    T xs[kU], ys[kU], zs[kU];
#if COMET_DCA_SCAN_P
                    T pxs[kU], pys[kU], pzs[kU];
#endif
#pragma unroll
                    for (int u = 0; u < kU; ++u) {
                        const int k = k0 + t0 + u;
                        xs[u] = ys[u] = zs[u] = T(0);
#if COMET_DCA_SCAN_P
                        pxs[u] = pys[u] = pzs[u] = T(0);
#endif
                        if (want && k < k1) {
                            const T *q = q0 + u * S;
                            xs[u] = q[0];
                            ys[u] = q[plane];
                            zs[u] = q[2 * plane];
#if COMET_DCA_SCAN_P
                            pxs[u] = q[3 * plane];
                            pys[u] = q[4 * plane];
                            pzs[u] = q[5 * plane];
#endif
                        }
                    }
#pragma unroll
                    for (int u = 0; u < kU; ++u) {
                        const int k = k0 + t0 + u;
                        if (want && k < k1) {
#if COMET_DCA_SCAN_P
                            const T d = sd2(xs[u], ys[u], zs[u]);
                            if (d < bd || (d == bd && k < bk)) {
                                bdm = k == kprev + 1 ? dprev : T(INFINITY);
                                bdp = T(INFINITY);
                                bd = d;
                                bk = k;
                                by[0] = xs[u];
                                by[1] = ys[u];
                                by[2] = zs[u];
                                by[3] = pxs[u];
                                by[4] = pys[u];
                                by[5] = pzs[u];
                            } else if (k == bk + 1) {
                                bdp = d;
                            }
                            dprev = d;
                            kprev = k;
#else
                            lex_min<T>(bd, bk, sd2(xs[u], ys[u], zs[u]), k);
#endif
                        }
                    }
                }
            };
            if (a.exact_all) {
                int nvw = nv;
#pragma unroll
                for (int off = 16; off > 0; off >>= 1) nvw = max(nvw, __shfl_xor_sync(0xffffffffu, nvw, off));
                scan(0, nv, nvw);
            } else {
                uint32_t u0 = m0;
                while (u0) {
                    const int j = __ffs(u0) - 1;
                    u0 &= u0 - 1;
                    // lane m tests level-1 segment m of super-segment j; a one-state segment
                    // that may hold a track end (the first state, or between the warp's smallest
                    // and largest last state) gets the refinement's extra half interval there
                    const int k1 = j * G0 + lane;
                    const bool end1 = G1 == 1 && (k1 == 0 || (k1 >= gr.elo && k1 <= gr.ehi));
                    // one-state segments away from the track ends need only the interior reach
                    const T lim1 = G1 == 1 ? (end1 ? capth + half_rec : thin) : capth;
                    bool hit1;
                    if constexpr (sizeof(T) == 8)
                        hit1 = lane < N1 &&
                               sphere_within<float>(sph1[j * kN1Max + lane], (float)fvx, (float)fvy,
                                                    (float)fvz, (float)fav, (float)fwx, (float)fwy,
                                                    (float)fwz, (float)faw, (float)ax, (float)ay,
                                                    (float)az, (float)ux, (float)uy, (float)uz,
                                                    (float)lim1 + sph_margin_f32(fav, faw));
                    else
                        hit1 = lane < N1 &&
                               sphere_within<T>(sph1[j * kN1Max + lane], fvx, fvy, fvz, fav, fwx, fwy,
                                                fwz, faw, ax, ay, az, ux, uy, uz, lim1);
                    const uint32_t u1 = __ballot_sync(0xffffffffu, hit1);
                    if (u1) {
                        // one contiguous range from the first to the last candidate level-1
                        // segment (a superset of the candidates; their loads go out together)
                        const int m_lo = __ffs(u1) - 1, m_hi = 31 - __clz(u1);
                        const int sb = j * G0, se = min(sb + G0, nv);
                        const int k0 = sb + m_lo * G1;
                        scan(k0, min(sb + (m_hi + 1) * G1, se), (m_hi - m_lo + 1) * G1);
                    }
                }
            }

            // refinement from the closest recorded state, only where it can bring the wire within
            // its capture radius: from an interior state within the interior reach thin, from the
            // first or the last recorded state within a whole interval more than capth (the
            // refinement may extrapolate h_rec beyond the track); compared squared: the thresholds
            // carry margins far above the rounding of the square
            const T th = (bk == 0 || bk == nv - 1) ? capth + half_rec : thin;
            const bool refine = want && bk != 0x7fffffff && (a.exact_all || bd <= th * th);
            T D = T(INFINITY);
            if (refine) {
                T yv[6];
                T s0 = T(0);
#if COMET_DCA_SCAN_P
#pragma unroll
                for (int cc = 0; cc < 6; ++cc) yv[cc] = by[cc];
                // first step to the vertex of the parabola through the squared distances of the
                // closest state and its two neighbours (exact for a straight track, where the
                // squared distance is quadratic in arc length); then Newton steps as usual.  Used
                // when both neighbours were scanned and the step budget allows (max_iter >= 4).
                if (a.max_iter >= 4 && bdm < T(INFINITY) && bdp < T(INFINITY)) {
                    const T den = bdm - T(2) * bd + bdp;
                    if (den > T(0)) {
                        s0 = T(0.5) * h_rec * (bdm - bdp) / den;
                        s0 = fmin(fmax(s0, -h_rec), h_rec);
                    }
                }
#else
                const int64_t o = (int64_t)bk * S + s;
#pragma unroll
                for (int cc = 0; cc < 6; ++cc) yv[cc] = P[cc * plane + o];
#endif
                const int conv = refine_dca<T, F>(f, gr.c, gr.ip, yv, ax, ay, az, ux, uy, uz, tol,
                                                  a.max_iter, h_rec, D, s0);
                if (cap >= T(0)) nunc += 1 - conv;
                if (a.dca_out) ((T *)a.dca_out)[(int64_t)(tl.w0 + ii) * S + s] = D;
            }
            if (valid && cap >= T(0)) {
                T emin = T(INFINITY);
                if (refine) {
                    const int hb = tl.offs[ii], he = tl.offs[ii + 1];
                    for (int j = hb; j < he; ++j) {
                        if (tl.msm[j]) continue;
                        const T e = fabs(D - tl.dsm[j]);
                        emin = e < emin ? e : emin;
                    }
                }
                const T d = emin < lam ? emin : lam;
                nin += emin < lam ? 1 : 0;
                acc.add(d * d);
            }
        }
    }
}

// Wire chunk c of n over W wires: [c * wc, min((c + 1) * wc, W)), wc = ceil(W / n).
__device__ __forceinline__ int2 chunk_range(int W, int n, int c)
{
    const int wc = (W + n - 1) / n;
    return make_int2(min(c * wc, W), min((c + 1) * wc, W));
}

// All wire chunks of one group in this warp: each chunk's partial sum, added in chunk order (the
// arithmetic the cross-warp schedule of the persistent kernel reproduces).
template <typename T, class F>
__device__ __forceinline__ void group_all_chunks(const F &f, const DcaArgs &a, const Group<T> &gr,
                                                 const Tile<T> &tl, const float4 *sph0,
                                                 const float4 *sph1, int lane, Acc<T> &acc,
                                                 int &nin, int &nunc)
{
    for (int c = 0; c < a.n_chunks; ++c) {
        const int2 r = chunk_range(tl.wn, a.n_chunks, c);
        Acc<T> part;
        group_wires<T, F>(f, a, gr, tl, sph0, sph1, lane, part, nin, nunc, r.x, r.y);
        acc.add_pair(part.hi, part.lo);
    }
}

// Waits for a staging transaction of `bytes` (thread 0 issued it; everyone waits) for at most
// wait_ns; wait_ns = 0 gives up at once without waiting (the context's test setting).  Returns true
// if the wait gave up anywhere in the CTA: the caller then re-reads the data with plain loads and,
// before its shared memory or barrier is used again, waits (up to kWaitNs) for the abandoned copy.
__device__ __forceinline__ bool finish_stage(uint64_t *bar, uint32_t &parity, uint32_t bytes,
                                             uint64_t wait_ns)
{
    bool to = false;
    if (bytes > 0) {
        to = wait_ns == 0 ? true : !mbar_wait(bar, parity, wait_ns);
        parity ^= 1u;
    }
    return __syncthreads_or(to);
}

// ------------------------------------------------------------------------------------------------
// The seed of lowest RSS, selected inside the DCA launch (optional; the k = 1 case of
// comet_scan_select, in its order: ascending RSS, NaN after every number, ties by lowest index).
// The warp that finalises a group folds the group's best into its warp's best (shared memory); at
// the end each CTA folds its warps into a slot, and the last CTA to finish folds the slots.
// ------------------------------------------------------------------------------------------------

template <typename T>
struct Best {
    T v;
    int64_t i;
};

template <typename T>
__device__ __forceinline__ T nan_value()
{
    if constexpr (sizeof(T) == 4)
        return __int_as_float(0x7fc00000);
    else
        return __longlong_as_double(0x7ff8000000000000ll);
}

template <typename T>
__device__ __forceinline__ Best<T> best_none()
{
    return Best<T>{nan_value<T>(), INT64_MAX};
}

// (v, i) before (b.v, b.i) in comet_scan_select's order
template <typename T>
__device__ __forceinline__ bool precedes(T v, int64_t i, const Best<T> &b)
{
    const bool vn = v != v, bn = b.v != b.v;
    if (vn != bn) return bn;
    if (!vn && v != b.v) return v < b.v;
    return i < b.i;
}

template <typename T>
__device__ __forceinline__ void best_fold(Best<T> &b, T v, int64_t i)
{
    if (precedes<T>(v, i, b)) {
        b.v = v;
        b.i = i;
    }
}

// The best of the warp's 32 candidates, in every lane.
template <typename T>
__device__ __forceinline__ Best<T> warp_best(Best<T> b)
{
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        const T v = __shfl_xor_sync(0xffffffffu, b.v, off);
        const int64_t i = __shfl_xor_sync(0xffffffffu, b.i, off);
        best_fold<T>(b, v, i);
    }
    return b;
}

// A finalised group: the best of its valid seeds folded into this warp's best (s_warp[warp]).
template <typename T>
__device__ __forceinline__ void group_best_fold(Best<T> *s_warp, int warp, int lane, bool valid, T rss,
                                                int64_t s)
{
    Best<T> b = valid ? Best<T>{rss, s} : best_none<T>();
    b = warp_best<T>(b);
    if (lane == 0) best_fold<T>(s_warp[warp], b.v, b.i);
}

// End of the launch (every thread of the CTA): the CTA's best into its slot; the last CTA to finish
// folds every slot and writes the selection, then leaves the counter at zero for the next launch.
template <typename T>
__device__ __forceinline__ void finish_best(const DcaArgs &a, Best<T> *s_warp, int *s_last)
{
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    int64_t *slot_i = (int64_t *)a.best_slots;
    T *slot_v = (T *)(slot_i + gridDim.x);
    __syncthreads();
    if (tid == 0) {
        Best<T> b = s_warp[0];
        for (int w = 1; w < kWarps; ++w) best_fold<T>(b, s_warp[w].v, s_warp[w].i);
        slot_i[blockIdx.x] = b.i;
        slot_v[blockIdx.x] = b.v;
        __threadfence();
        const unsigned int t = atomicAdd(a.best_counter, 1u);
        *s_last = t == gridDim.x - 1;
    }
    __syncthreads();
    if (*s_last) {
        __threadfence();
        Best<T> b = best_none<T>();
        for (unsigned int k = tid; k < gridDim.x; k += blockDim.x) best_fold<T>(b, __ldcg(slot_v + k), __ldcg(slot_i + k));
        b = warp_best<T>(b);
        if (lane == 0) s_warp[warp] = b;
        __syncthreads();
        if (tid == 0) {
            Best<T> r = s_warp[0];
            for (int w = 1; w < kWarps; ++w) best_fold<T>(r, s_warp[w].v, s_warp[w].i);
            *a.best_idx_out = r.i;
            if (a.best_rss_out) *(T *)a.best_rss_out = r.v;
            *a.best_counter = 0u;
        }
    }
}

// ------------------------------------------------------------------------------------------------
// Persistent kernel: all wires fit one shared-memory tile (the common case).  Each CTA stages the
// wires and hits once; each warp then takes work items -- (32-seed group, wire chunk) pairs, or
// whole groups when no partial-sum scratch is given -- from a device counter until none is left,
// with no CTA-wide barrier between items.
// ------------------------------------------------------------------------------------------------

struct PLayout {
    size_t sph, wrow, orow, cap, frame, drift, mask, total;
    int wcap;
    int nsph;    // float4 sphere entries per warp
};

// Sphere entries each warp keeps in shared memory: the whole table (built here) when no bounds
// table was given; with the recording kernel's table, the part a group can use -- its kN0Max
// super-segment spheres and the level-1 spheres of the super-segments an n_rec-state track has --
// copied in per work item (about 1.3 KB per warp at 70 recorded states, so that the per-wire
// level-1 tests read shared memory, not L2); none when every state is scanned (dca_out requested).
__host__ __device__ inline int p_sph_entries(const DcaArgs &a)
{
    if (a.exact_all) return 0;
    if (a.bounds == nullptr) return kBoundsPerGroup;
    int n0 = (a.n_rec + a.G0 - 1) / a.G0;
    n0 = n0 < kN0Max ? n0 : kN0Max;
    return kN0Max + n0 * kN1Max;
}

__host__ __device__ inline PLayout p_layout(int W, int es, int nsph)
{
    PLayout L;
    int wc = ((W + 31) / 32) * 32;
    wc = wc < 32 ? 32 : wc;
    L.wcap = wc;
    L.nsph = nsph;
    L.sph = 16;
    L.wrow = align16(L.sph + (size_t)16 * kWarps * nsph);
    L.orow = align16(L.wrow + (size_t)es * 6 * (wc + 32));
    L.cap = align16(L.orow + (size_t)4 * (wc + 40));
    L.frame = align16(L.cap + (size_t)es * wc);
    L.drift = align16(L.frame + (size_t)es * 16 * wc);
    L.mask = align16(L.drift + (size_t)es * kHitCap);
    L.total = align16(L.mask + kHitCap);
    return L;
}

constexpr int kPersistMaxW = 1024;

template <typename T, class F>
__global__ void __launch_bounds__(kThreads, sizeof(T) == 8 ? COMET_DCA_MINB_F64 : (F::kAxial ? COMET_DCA_MINB : COMET_DCA_MINB_FIELD)) dca_persistent_kernel(F f, DcaArgs a)
{
    const bool sph_smem = a.bounds == nullptr && !a.exact_all;
    const PLayout L = p_layout(a.W, (int)sizeof(T), p_sph_entries(a));
    extern __shared__ __align__(128) unsigned char sm[];
    uint64_t *bar = (uint64_t *)sm;
    const int tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    float4 *sph0 = (float4 *)(sm + L.sph) + warp * L.nsph;
    float4 *sph1 = sph0 + kN0Max;
    T *wrow = (T *)(sm + L.wrow);
    int32_t *orow = (int32_t *)(sm + L.orow);
    T *capv = (T *)(sm + L.cap);
    Q4<T> *frm = (Q4<T> *)(sm + L.frame);
    T *dsm = (T *)(sm + L.drift);
    uint8_t *msm = (uint8_t *)(sm + L.mask);
    const int rcap = L.wcap + 32;
    const T *__restrict__ Wg = (const T *)a.wires;
    const T *__restrict__ Dg = (const T *)a.drift;
    const int W = a.W;
    const int H = W > 0 ? a.offs[W] : 0;
    const bool hits_sm = H <= kHitMax;
    __shared__ Best<T> s_best[kWarps];
    __shared__ int s_last;

    if (tid == 0) mbar_init(bar, 1);
    if (lane == 0) s_best[warp] = best_none<T>();
    __syncthreads();

    // ---- stage wires, offsets and (when they fit) hits: one bulk-copy transaction (W > 0 only:
    // with no wires the pointers may be NULL and every RSS is 0)
    uint32_t parity = 0;
    uint32_t bytes = 0;
    int woff[6] = {0, 0, 0, 0, 0, 0};
    int ooff = 0, doff = 0, moff = 0;
    if (W > 0) {
        bytes = stage_bytes<int32_t>(a.offs, W + 1);
#pragma unroll
        for (int r = 0; r < 6; ++r) bytes += stage_bytes<T>(Wg + (size_t)r * a.ldw, W);
        if (hits_sm && H > 0) bytes += stage_bytes<T>(Dg, H) + stage_bytes<uint8_t>(a.mask, H);
        if (tid == 0 && bytes > 0) {
            fence_proxy_async_smem();
            mbar_arrive_expect_tx(bar, bytes);
        }
#pragma unroll
        for (int r = 0; r < 6; ++r)
            woff[r] = stage_issue<T>(wrow + r * rcap, Wg + (size_t)r * a.ldw, W, bar, tid == 0);
        ooff = stage_issue<int32_t>(orow, a.offs, W + 1, bar, tid == 0);
        if (hits_sm && H > 0) {
            doff = stage_issue<T>(dsm, Dg, H, bar, tid == 0);
            moff = stage_issue<uint8_t>(msm, a.mask, H, bar, tid == 0);
        }
    }
    const bool any_timeout = finish_stage(bar, parity, bytes, a.wait_ns);
    if (any_timeout && W > 0) {
#pragma unroll
        for (int r = 0; r < 6; ++r) stage_fallback<T>(wrow + r * rcap, Wg + (size_t)r * a.ldw, W);
        stage_fallback<int32_t>(orow, a.offs, W + 1);
        if (hits_sm && H > 0) {
            stage_fallback<T>(dsm, Dg, H);
            stage_fallback<uint8_t>(msm, a.mask, H);
        }
    }
    __syncthreads();
    Tile<T> tl;
    tl.ax = wrow + 0 * rcap + woff[0];
    tl.ay = wrow + 1 * rcap + woff[1];
    tl.az = wrow + 2 * rcap + woff[2];
    tl.ux = wrow + 3 * rcap + woff[3];
    tl.uy = wrow + 4 * rcap + woff[4];
    tl.uz = wrow + 5 * rcap + woff[5];
    tl.rec = frm;
    tl.cap = capv;
    tl.offs = orow + ooff;
    tl.dsm = hits_sm ? dsm + doff : Dg;
    tl.msm = hits_sm ? msm + moff : a.mask;
    tl.w0 = 0;
    tl.wn = W;
    for (int i = tid; i < W; i += kThreads) tile_wire_setup<T>(tl, i, in_prec<T>(a.lambda, a.lambda_f), capv, frm);
    __syncthreads();

    // ---- work items taken dynamically by each warp: 32-seed groups, or (group, wire chunk) pairs
    // when partial sums can be parked in `part` (finer items balance the warps' loads)
    const int64_t n_groups = (a.S + 31) / 32;
    const bool split = a.n_chunks > 1 && a.part && a.arrive;
    const int nc = split ? a.n_chunks : 1;
    const int64_t n_items = n_groups * nc;
    int nunc = 0;
    for (;;) {
        unsigned int it = 0;
        if (lane == 0) it = atomicAdd((unsigned int *)a.counter, 1u);
        it = __shfl_sync(0xffffffffu, it, 0);
        if ((int64_t)it >= n_items) break;
        const int64_t g = (int64_t)(it / (unsigned)nc);
        const int c = (int)(it % (unsigned)nc);
        const Group<T> gr = load_group<T>(a, g, lane);
        if (sph_smem) {
            build_spheres<T>(a, gr, lane, sph0, sph1, g);
        } else if (L.nsph > 0) {
            // the usable part of this group's table from the recording kernel
            const float4 *src = (const float4 *)a.bounds + g * kBoundsPerGroup;
            for (int i = lane; i < L.nsph; i += 32) sph0[i] = __ldg(src + i);
            __syncwarp();
        }
        const float4 *s0 = sph0, *s1 = sph1;
        Acc<T> acc;
        int nin = 0;
        if (!split) {
            group_all_chunks<T, F>(f, a, gr, tl, s0, s1, lane, acc, nin, nunc);
            const T v = acc.value();
            if (gr.valid) {
                ((T *)a.rss)[gr.s] = v;
                a.n_in[gr.s] = nin;
            }
            if (a.best_idx_out) group_best_fold<T>(s_best, warp, lane, gr.valid, v, gr.s);
        } else {
            const int2 r = chunk_range(W, nc, c);
            group_wires<T, F>(f, a, gr, tl, s0, s1, lane, acc, nin, nunc, r.x, r.y);
            T *ph = (T *)a.part;
            T *pl = ph + (size_t)nc * a.S;
            int32_t *pn = (int32_t *)(pl + (size_t)nc * a.S);
            if (gr.valid) {
                ph[(int64_t)c * a.S + gr.s] = acc.hi;
                pl[(int64_t)c * a.S + gr.s] = acc.lo;
                pn[(int64_t)c * a.S + gr.s] = nin;
            }
            __threadfence();
            __syncwarp();
            unsigned int done = 0;
            if (lane == 0) done = atomicAdd(a.arrive + g, 1u);
            done = __shfl_sync(0xffffffffu, done, 0);
            if (done == (unsigned)(nc - 1)) {
                // the group's last chunk: add the partial sums in chunk order
                __threadfence();
                T v = T(0);
                if (gr.valid) {
                    Acc<T> tot;
                    int nt = 0;
                    for (int k = 0; k < nc; ++k) {
                        const int64_t o = (int64_t)k * a.S + gr.s;
                        tot.add_pair(__ldcg(ph + o), __ldcg(pl + o));
                        nt += __ldcg(pn + o);
                    }
                    v = tot.value();
                    ((T *)a.rss)[gr.s] = v;
                    a.n_in[gr.s] = nt;
                }
                if (a.best_idx_out) group_best_fold<T>(s_best, warp, lane, gr.valid, v, gr.s);
                if (lane == 0) a.arrive[g] = 0u;   // left zero for the next launch
            }
        }
        __syncwarp();   // the next group's spheres overwrite this warp's slot
    }
    if (a.n_unconv) {
        int t = nunc;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) t += __shfl_xor_sync(0xffffffffu, t, off);
        if (lane == 0 && t) atomicAdd(a.n_unconv, t);
    }
    if (a.best_idx_out) finish_best<T>(a, s_best, &s_last);
    if (any_timeout) {
        if (tid == 0 && a.status) atomicOr(a.status, 1);
        mbar_wait(bar, parity ^ 1u, kWaitNs);
    }
}

// ------------------------------------------------------------------------------------------------
// Tiled kernel: more wires than one tile holds.  One 128-seed block per CTA; wires staged in tiles.
// ------------------------------------------------------------------------------------------------

template <typename T, class F>
__global__ void __launch_bounds__(kThreads, sizeof(T) == 8 ? COMET_DCA_MINB_F64 : (F::kAxial ? COMET_DCA_MINB : COMET_DCA_MINB_FIELD)) dca_tiled_kernel(F f, DcaArgs a)
{
    using L = Smem<T>;
    extern __shared__ __align__(128) unsigned char sm[];
    uint64_t *bar = (uint64_t *)(sm + L::bar);
    const int tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    float4 *sph0 = (float4 *)(sm + L::sph0) + warp * kN0Max;
    float4 *sph1 = (float4 *)(sm + L::sph1) + warp * kN0Max * kN1Max;
    T *wrow = (T *)(sm + L::wrow);
    int32_t *orow = (int32_t *)(sm + L::orow);
    T *capv = (T *)(sm + L::cap);
    Q4<T> *frm = (Q4<T> *)(sm + L::frame);
    T *dsm = (T *)(sm + L::drift);
    uint8_t *msm = (uint8_t *)(sm + L::mask);
    const T *__restrict__ Wg = (const T *)a.wires;
    const T *__restrict__ Dg = (const T *)a.drift;

    if (tid == 0) mbar_init(bar, 1);
    const int64_t g = (int64_t)blockIdx.x * kWarps + warp;
    const Group<T> gr = load_group<T>(a, g, lane);
    if (!a.exact_all) build_spheres<T>(a, gr, lane, sph0, sph1, g);

    const int W = a.W;
    const int H = W > 0 ? a.offs[W] : 0;
    const bool hits_sm = H <= kHitMax;
    uint32_t parity = 0;
    bool any_timeout = false;
    int doff = 0, moff = 0;
    __syncthreads();   // barrier initialised

    if (hits_sm && H > 0) {
        const uint32_t bytes = stage_bytes<T>(Dg, H) + stage_bytes<uint8_t>(a.mask, H);
        if (tid == 0 && bytes > 0) {
            fence_proxy_async_smem();
            mbar_arrive_expect_tx(bar, bytes);
        }
        doff = stage_issue<T>(dsm, Dg, H, bar, tid == 0);
        moff = stage_issue<uint8_t>(msm, a.mask, H, bar, tid == 0);
        if (finish_stage(bar, parity, bytes, a.wait_ns)) {
            any_timeout = true;
            stage_fallback<T>(dsm, Dg, H);
            stage_fallback<uint8_t>(msm, a.mask, H);
            // the barrier is reused by the wire tiles: let the abandoned copy land first (bounded)
            mbar_wait(bar, parity ^ 1u, kWaitNs);
        }
        __syncthreads();
    }

    Acc<T> acc;
    int nin = 0, nunc = 0;
    for (int w0 = 0; w0 < W; w0 += kWireTile) {
        const int wn = min(kWireTile, W - w0);
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
        if (finish_stage(bar, parity, bytes, a.wait_ns)) {
            any_timeout = true;
#pragma unroll
            for (int r = 0; r < 6; ++r)
                stage_fallback<T>(wrow + r * kWireCap, Wg + (size_t)r * a.ldw + w0, wn);
            stage_fallback<int32_t>(orow, a.offs + w0, wn + 1);
            // the next tile reuses these buffers and the barrier: let the abandoned copy land
            // first (bounded)
            mbar_wait(bar, parity ^ 1u, kWaitNs);
        }
        __syncthreads();
        Tile<T> tl;
        tl.ax = wrow + 0 * kWireCap + woff[0];
        tl.ay = wrow + 1 * kWireCap + woff[1];
        tl.az = wrow + 2 * kWireCap + woff[2];
        tl.ux = wrow + 3 * kWireCap + woff[3];
        tl.uy = wrow + 4 * kWireCap + woff[4];
        tl.uz = wrow + 5 * kWireCap + woff[5];
        tl.rec = frm;
        tl.cap = capv;
        tl.offs = orow + ooff;
        tl.dsm = hits_sm ? dsm + doff : Dg;
        tl.msm = hits_sm ? msm + moff : a.mask;
        tl.w0 = w0;
        tl.wn = wn;
        for (int i = tid; i < wn; i += kThreads) tile_wire_setup<T>(tl, i, in_prec<T>(a.lambda, a.lambda_f), capv, frm);
        __syncthreads();
        group_wires<T, F>(f, a, gr, tl, sph0, sph1, lane, acc, nin, nunc, 0, wn);
        if (w0 + kWireTile < W) __syncthreads();   // tile consumed before the next staging
    }

    const T v = acc.value();
    if (gr.valid) {
        ((T *)a.rss)[gr.s] = v;
        a.n_in[gr.s] = nin;
    }
    if (a.n_unconv) {
        int t = nunc;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) t += __shfl_xor_sync(0xffffffffu, t, off);
        if (lane == 0 && t) atomicAdd(a.n_unconv, t);
    }
    if (a.best_idx_out) {
        __shared__ Best<T> s_best[kWarps];
        __shared__ int s_last;
        if (lane == 0) s_best[warp] = best_none<T>();
        __syncwarp();
        group_best_fold<T>(s_best, warp, lane, gr.valid, v, gr.s);
        finish_best<T>(a, s_best, &s_last);
    }
    if (any_timeout && tid == 0 && a.status) atomicOr(a.status, 1);
}

static int sm_count()
{
    static int n = [] {
        int dev = 0, v = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
        return v > 0 ? v : 1;
    }();
    return n;
}

template <typename T, class F>
static cudaError_t dca_launch(const F &fld, const DcaArgs &a, cudaStream_t st)
{
    if (a.W <= kPersistMaxW && a.counter) {
        const PLayout L = p_layout(a.W, (int)sizeof(T), p_sph_entries(a));
        cudaError_t e = cudaFuncSetAttribute(dca_persistent_kernel<T, F>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.total);
        if (e != cudaSuccess) return e;
        int per_sm = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, dca_persistent_kernel<T, F>,
                                                          kThreads, L.total);
        if (e != cudaSuccess) return e;
        per_sm = per_sm < 1 ? 1 : per_sm;
        if (a.max_ctas_per_sm > 0 && a.max_ctas_per_sm < per_sm) per_sm = a.max_ctas_per_sm;
        const int64_t items = (a.S + 31) / 32 * ((a.part && a.arrive) ? a.n_chunks : 1);
        int64_t nb = (items + kWarps - 1) / kWarps;
        const int64_t cap = (int64_t)per_sm * sm_count();
        nb = nb < cap ? nb : cap;
        e = cudaMemsetAsync(a.counter, 0, sizeof(int32_t), st);
        if (e != cudaSuccess) return e;
        if (a.best_idx_out && nb > a.best_slots_cap) return cudaErrorInvalidValue;   // one slot per CTA
        dca_persistent_kernel<T, F><<<(unsigned)nb, kThreads, L.total, st>>>(fld, a);
        return cudaGetLastError();
    }
    using L = Smem<T>;
    static const cudaError_t attr = cudaFuncSetAttribute(
        dca_tiled_kernel<T, F>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L::total);
    if (attr != cudaSuccess) return attr;
    const int64_t nb = (a.S + kThreads - 1) / kThreads;
    if (a.best_idx_out && nb > a.best_slots_cap) return cudaErrorInvalidValue;   // one slot per CTA
    dca_tiled_kernel<T, F><<<(unsigned)nb, kThreads, L::total, st>>>(fld, a);
    return cudaGetLastError();
}

template <typename T>
static cudaError_t dca_dispatch(const comet_field &f, const DcaArgs &a, cudaStream_t st)
{
    switch (field_kind(f)) {
    case FieldKind::Axial:
        return dca_launch<T>(FieldAxial<T>{(T)f.b[2]}, a, st);
    case FieldKind::Uniform:
        return dca_launch<T>(FieldUniform<T>{(T)f.b[0], (T)f.b[1], (T)f.b[2]}, a, st);
    case FieldKind::Table:
    default:
        return dca_launch<T>(make_table<T>(f),
                             a, st);
    }
}

int dca_wire_chunks(int W, int64_t S, int chunk_wires)
{
    if (W <= 0 || W > kPersistMaxW) return 1;
    if (chunk_wires > 0) {
        // a fixed width (the context's setting), at most kDcaBatchSub chunks
        const int n = (W + chunk_wires - 1) / chunk_wires;
        return n < kDcaBatchSub ? n : kDcaBatchSub;
    }
    int nc = (W + COMET_DCA_CHUNK_W - 1) / COMET_DCA_CHUNK_W;
    // few seeds: narrower chunks (at least 4 wires, at most kDcaBatchSub of them), so that the
    // (32-seed group, chunk) work items occupy every SM
    constexpr int64_t kTargetItems = 4096;
    const int64_t groups = (S + 31) / 32;
    if (groups > 0 && groups * nc < kTargetItems) {
        const int64_t want = (kTargetItems + groups - 1) / groups;
        int cap = W / 4;
        cap = cap < kDcaBatchSub ? cap : kDcaBatchSub;
        if (want > nc && cap > nc) nc = (int)(want < cap ? want : cap);
    }
    return nc;
}

void dca_segments(int n_rec, int *G0, int *G1)
{
    if (n_rec <= kN0Max * kN1Max) {
        // one state per level-1 segment: its sphere is then just the spread of the group's tracks
        const int n0 = (n_rec + kN1Max - 1) / kN1Max;
        *G0 = (n_rec + n0 - 1) / n0;
        *G1 = 1;
        return;
    }
    // up to 8 super-segments, each cut into level-1 segments of 3 states (more when a super-segment
    // would have more than kN1Max of them)
    int n0 = (int)lround(cbrt((double)n_rec));
    n0 = n0 < 1 ? 1 : (n0 > kN0Max ? kN0Max : n0);
    const int g0 = (n_rec + n0 - 1) / n0;
    int g1 = 3;
    if ((g0 + g1 - 1) / g1 > kN1Max) g1 = (g0 + kN1Max - 1) / kN1Max;
    *G0 = g0;
    *G1 = g1 > g0 ? g0 : g1;
}

// ------------------------------------------------------------------------------------------------
// Batch of events: persistent CTAs take items -- dca_batch_groups(n_chunks) consecutive 32-seed
// groups of one event -- from ONE counter over all events (items numbered event by event,
// BL.dca_start the prefix), so the load balances across events as it does in the single-event
// kernel.  Inside an item the warps share out its (group, wire chunk) sub-items from a shared
// counter, park the partial sums in the CTA's slice of BL.dca_part, and add them per seed in chunk
// order once the item is done (the single-event kernel's arithmetic).  A CTA restages wires and
// hits only when its next item belongs to another event (a few KB by bulk copy).  Shared memory is
// laid out for the batch's largest W.
// ------------------------------------------------------------------------------------------------

#ifndef COMET_DCA_BATCH_MINB
#define COMET_DCA_BATCH_MINB 6   // the event's arguments come from a table, not the parameter bank
#endif

template <typename T, class F>
__global__ void __launch_bounds__(kThreads, COMET_DCA_BATCH_MINB) dca_batch_kernel(F f, BatchLaunch BL)
{
    const PLayout L = p_layout(BL.W_max, (int)sizeof(T), 0);   // batches read their bounds in place
    extern __shared__ __align__(128) unsigned char sm[];
    uint64_t *bar = (uint64_t *)sm;
    __shared__ int64_t s_chunk;
    __shared__ int s_sub;
    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const int warp = tid >> 5;
    T *wrow = (T *)(sm + L.wrow);
    int32_t *orow = (int32_t *)(sm + L.orow);
    T *capv = (T *)(sm + L.cap);
    Q4<T> *frm = (Q4<T> *)(sm + L.frame);
    T *dsm = (T *)(sm + L.drift);
    uint8_t *msm = (uint8_t *)(sm + L.mask);
    const int rcap = L.wcap + 32;
    if (tid == 0) mbar_init(bar, 1);
    __syncthreads();

    const int64_t n_chunks = BL.dca_start[BL.B];
    uint32_t parity = 0;
    bool timed_out = false;
    int cur = -1;
    // the current event's arguments and staged tile live in shared memory (they change only on a
    // restage): registers stay free for the group loop
    __shared__ DcaArgs s_a;
    __shared__ Tile<T> s_tl;
    const DcaArgs &a = s_a;
    const Tile<T> &tl = s_tl;
    int nunc = 0;
    for (;;) {
        if (tid == 0) {
            s_chunk = (int64_t)atomicAdd((unsigned long long *)BL.chunk_counter, 1ull);
            s_sub = 0;
        }
        __syncthreads();
        const int64_t chunk = s_chunk;
        if (chunk >= n_chunks) break;
        int e;
        int64_t lc;
        batch_find(BL.dca_start, BL.B, chunk, e, lc);
        if (e != cur) {
            // flush this CTA's unconverged count to the event it leaves
            if (cur >= 0 && a.n_unconv) {
                int t = nunc;
#pragma unroll
                for (int off = 16; off > 0; off >>= 1) t += __shfl_xor_sync(0xffffffffu, t, off);
                if (lane == 0 && t) atomicAdd(a.n_unconv, t);
            }
            nunc = 0;
            // every thread is past its last use of s_a / s_tl (the barrier closing the chunk)
            if (tid == 0) s_a = BL.ev[e].dca;
            __syncthreads();
            cur = e;
            const T *__restrict__ Wg = (const T *)a.wires;
            const T *__restrict__ Dg = (const T *)a.drift;
            const int W = a.W;
            const int H = W > 0 ? a.offs[W] : 0;
            const bool hits_sm = H <= kHitMax;
            // every thread's earlier shared-memory accesses before the bulk copies overwrite them
            fence_proxy_async_smem();
            __syncthreads();
            uint32_t bytes = 0;
            int woff[6] = {0, 0, 0, 0, 0, 0};
            int ooff = 0, doff = 0, moff = 0;
            if (W > 0) {
                bytes = stage_bytes<int32_t>(a.offs, W + 1);
#pragma unroll
                for (int r = 0; r < 6; ++r) bytes += stage_bytes<T>(Wg + (size_t)r * a.ldw, W);
                if (hits_sm && H > 0) bytes += stage_bytes<T>(Dg, H) + stage_bytes<uint8_t>(a.mask, H);
                if (tid == 0 && bytes > 0) mbar_arrive_expect_tx(bar, bytes);
#pragma unroll
                for (int r = 0; r < 6; ++r)
                    woff[r] = stage_issue<T>(wrow + r * rcap, Wg + (size_t)r * a.ldw, W, bar, tid == 0);
                ooff = stage_issue<int32_t>(orow, a.offs, W + 1, bar, tid == 0);
                if (hits_sm && H > 0) {
                    doff = stage_issue<T>(dsm, Dg, H, bar, tid == 0);
                    moff = stage_issue<uint8_t>(msm, a.mask, H, bar, tid == 0);
                }
            }
            const bool to = finish_stage(bar, parity, bytes, a.wait_ns);
            if (to && W > 0) {
#pragma unroll
                for (int r = 0; r < 6; ++r) stage_fallback<T>(wrow + r * rcap, Wg + (size_t)r * a.ldw, W);
                stage_fallback<int32_t>(orow, a.offs, W + 1);
                if (hits_sm && H > 0) {
                    stage_fallback<T>(dsm, Dg, H);
                    stage_fallback<uint8_t>(msm, a.mask, H);
                }
            }
            if (to) {
                // a timed-out copy may still land: wait for it (bounded) before anything reuses
                // the buffers, and report it
                timed_out = true;
                if (tid == 0 && a.status) atomicOr(a.status, 1);
                mbar_wait(bar, parity ^ 1u, kWaitNs);
            }
            if (tid == 0) {
                s_tl.ax = wrow + 0 * rcap + woff[0];
                s_tl.ay = wrow + 1 * rcap + woff[1];
                s_tl.az = wrow + 2 * rcap + woff[2];
                s_tl.ux = wrow + 3 * rcap + woff[3];
                s_tl.uy = wrow + 4 * rcap + woff[4];
                s_tl.uz = wrow + 5 * rcap + woff[5];
                s_tl.rec = frm;
                s_tl.cap = capv;
                s_tl.offs = orow + ooff;
                s_tl.dsm = hits_sm ? dsm + doff : Dg;
                s_tl.msm = hits_sm ? msm + moff : a.mask;
                s_tl.w0 = 0;
                s_tl.wn = W;
            }
            __syncthreads();
            for (int i = tid; i < W; i += kThreads) tile_wire_setup<T>(tl, i, in_prec<T>(a.lambda, a.lambda_f), capv, frm);
            __syncthreads();
        }
        // the item's (group, wire chunk) sub-items, taken by the warps as they come free
        const int nc = a.n_chunks;
        const int64_t n_groups = (a.S + 31) / 32;
        const int gpi = a.batch_groups > 0 ? a.batch_groups : dca_batch_groups(nc);
        const int64_t g0 = lc * gpi;
        const int ng = (int)min((int64_t)gpi, n_groups - g0);
        const int n_sub = ng * nc;
        T *ph = (T *)((unsigned char *)BL.dca_part +
                      (size_t)blockIdx.x * kDcaBatchSub * 32 * (2 * sizeof(T) + 4));
        T *pl = ph + kDcaBatchSub * 32;
        int32_t *pn = (int32_t *)(pl + kDcaBatchSub * 32);
        for (;;) {
            int k = 0;
            if (lane == 0) k = atomicAdd(&s_sub, 1);
            k = __shfl_sync(0xffffffffu, k, 0);
            if (k >= n_sub) break;
            const int64_t g = g0 + k / nc;
            const Group<T> gr = load_group<T>(a, g, lane);
            const float4 *s0 = (const float4 *)a.bounds + g * kBoundsPerGroup;   // read in place
            Acc<T> acc;
            int nin = 0;
            const int2 r = chunk_range(a.W, nc, k % nc);
            group_wires<T, F>(f, a, gr, tl, s0, s0 + kN0Max, lane, acc, nin, nunc, r.x, r.y);
            ph[k * 32 + lane] = acc.hi;
            pl[k * 32 + lane] = acc.lo;
            pn[k * 32 + lane] = nin;
        }
        __syncthreads();   // every sub-item of the item done (and its partial sums visible)
        for (int gi = warp; gi < ng; gi += kWarps) {
            const int64_t s = (g0 + gi) * 32 + lane;
            if (s < a.S) {
                Acc<T> tot;
                int nt = 0;
                for (int c = 0; c < nc; ++c) {
                    const int k = (gi * nc + c) * 32 + lane;
                    tot.add_pair(ph[k], pl[k]);
                    nt += pn[k];
                }
                ((T *)a.rss)[s] = tot.value();
                a.n_in[s] = nt;
            }
        }
        __syncthreads();   // every warp done with this item before a restage or the next s_chunk
    }
    if (cur >= 0 && a.n_unconv) {
        int t = nunc;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) t += __shfl_xor_sync(0xffffffffu, t, off);
        if (lane == 0 && t) atomicAdd(a.n_unconv, t);
    }
    (void)timed_out;
}

template <typename T, class F>
static cudaError_t dca_batch_launch(const F &fld, const BatchLaunch &BL, cudaStream_t st)
{
    // (the shared-memory attribute for W_max was set when the batch was prepared: nothing here but
    // stream work, so that the launch can be captured)
    const PLayout L = p_layout(BL.W_max, (int)sizeof(T), 0);
    cudaError_t e = cudaMemsetAsync(BL.chunk_counter, 0, sizeof(unsigned long long), st);
    if (e != cudaSuccess) return e;
    if (BL.dca_ctas == 0) return cudaSuccess;
    dca_batch_kernel<T, F><<<BL.dca_ctas, kThreads, L.total, st>>>(fld, BL);
    return cudaGetLastError();
}

template <typename T, class F>
static int dca_ctas_per_sm_t(int W)
{
    const PLayout L = p_layout(W, (int)sizeof(T), 0);
    if (cudaFuncSetAttribute(dca_batch_kernel<T, F>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)L.total) != cudaSuccess)
        return 0;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, dca_batch_kernel<T, F>, kThreads,
                                                      L.total) != cudaSuccess)
        return 0;
    return per_sm;
}

template <typename T>
static int dca_ctas_per_sm_field(const comet_field &f, int W)
{
    switch (field_kind(f)) {
    case FieldKind::Axial: return dca_ctas_per_sm_t<T, FieldAxial<T>>(W);
    case FieldKind::Uniform: return dca_ctas_per_sm_t<T, FieldUniform<T>>(W);
    default: return dca_ctas_per_sm_t<T, FieldTable<T>>(W);
    }
}

int dca_persistent_ctas_per_sm(comet_dtype dt, const comet_field &f, int W)
{
    return dt == COMET_F32 ? dca_ctas_per_sm_field<float>(f, W) : dca_ctas_per_sm_field<double>(f, W);
}

int device_sm_count() { return sm_count(); }

template <typename T>
static cudaError_t dca_batch_dispatch(const comet_field &f, const BatchLaunch &BL, cudaStream_t st)
{
    switch (field_kind(f)) {
    case FieldKind::Axial:
        return dca_batch_launch<T>(FieldAxial<T>{(T)f.b[2]}, BL, st);
    case FieldKind::Uniform:
        return dca_batch_launch<T>(FieldUniform<T>{(T)f.b[0], (T)f.b[1], (T)f.b[2]}, BL, st);
    case FieldKind::Table:
    default:
        return dca_batch_launch<T>(make_table<T>(f),
                                   BL, st);
    }
}

cudaError_t launch_dca_batch(comet_dtype dt, const comet_field &f, const BatchLaunch &BL, cudaStream_t st)
{
    return dt == COMET_F32 ? dca_batch_dispatch<float>(f, BL, st) : dca_batch_dispatch<double>(f, BL, st);
}

cudaError_t launch_dca(comet_dtype dt, const comet_field &f, const DcaArgs &a, cudaStream_t st)
{
    return dt == COMET_F32 ? dca_dispatch<float>(f, a, st) : dca_dispatch<double>(f, a, st);
}

} // namespace comet
