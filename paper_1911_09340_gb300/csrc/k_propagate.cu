// Seed lattice and track recording (Algorithm 1, Sec. 2.2.1).
//
// propagate_kernel: one thread extrapolates one seed with fixed-step RK4 and writes every
// stride-th state to the SoA track array points[c][k][s] (seed index fastest, so the 32 lanes of a
// warp store 32 consecutive values of one component: full 128-byte lines).  In a uniform axial field
// one RK4 step is a linear map (device.cuh), so a recording interval of `stride` steps is the
// product of `stride` such maps, formed once per seed in double and applied once per record.
// Steps after the last recorded state (n_steps not a multiple of stride) cannot change any output
// and are not taken.  Optionally the kernel also writes the bounding spheres of the track segments
// of each group of 32 consecutive seeds (one warp), which the DCA kernel's closest-state search
// uses: the 32 lanes record state r together, so a segment's sphere is one warp reduction at the
// moment its centre state is recorded.  The FP32 path keeps every state component as an
// unevaluated float pair (hi, lo) updated with TwoSum (Fast2Sum for the axial interval map, see
// device.cuh), so that the rounding of 6,500 steps does not accumulate (plain FP32 drifts ~0.1 mm
// over three turns; the pair stays within ~0.3 um of FP64).  The step maps read the leading float
// only.
#include "device.cuh"
#include "internal.h"

namespace comet {

// Seed s of the lattice: blocks of b = (2, 4, 4, 1) nodes along (z0, phi, pz, pt) (2 for phi or pz
// when only 2 divides the count, 1 when it is odd) numbered row-major, nodes inside a block
// row-major.  Consecutive seeds are therefore lattice neighbours of one pT, so the 32 lanes of a
// warp follow similar tracks in the DCA kernel (a pT step moves a track ~8 mm by the end of a turn,
// a phi or pz step ~3-4 mm).
// Node value i of a dimension with n nodes (computed in double with rounded operations only, so
// that it equals the oracle's value).
__device__ __forceinline__ double lattice_node(double centre, double half_width, int n, int i)
{
    return n == 1 ? centre
                  : __dadd_rn(centre, __dmul_rn(half_width, __dadd_rn(__ddiv_rn(2.0 * i, (double)(n - 1)), -1.0)));
}

constexpr int kLatTab = 512;   // node values tabulated per block when the four counts sum to <= this

// Grid (blocks, K): row k of the grid writes lattice k, seeds [k*S1, (k+1)*S1).  With refs == NULL
// there is one lattice centred at a.centre; otherwise lattice k is centred at refs[k'] (4 doubles:
// z0, phi, pz, pt), k' = k while k < *n_refs, else 0 (a repeat of the first, so that the seed count
// stays fixed whatever the number of references found).
// BATCH: one launch for the lattices of a batch of events; block b belongs to the event that
// batch_find gives (refs unused).
template <typename T, bool BATCH>
__global__ void __launch_bounds__(256) lattice_kernel(LatArgs a, const __grid_constant__ LatTable lt,
                                                      const double *__restrict__ refs,
                                                      const int32_t *__restrict__ n_refs,
                                                      T *__restrict__ seeds, int64_t S1, int64_t S,
                                                      BatchLaunch L)
{
    // the host's table of node values and phi-node cos / sin when there is one (lt, read in place,
    // or the batch event's copy); otherwise every node value (and cos / sin of every phi node)
    // once per block, in shared memory
    __shared__ double nodes[kLatTab];
    __shared__ double cphi[kLatTab], sphi[kLatTab];
    int64_t bx = blockIdx.x;
    const LatTable *tp = (!BATCH && lt.use && !refs) ? &lt : nullptr;
    if constexpr (BATCH) {
        int e;
        int64_t lb;
        if (!batch_find(L.lat_start, L.B, blockIdx.x, e, lb)) return;
        a = L.ev[e].lat;
        tp = L.ev[e].lat_tab.use ? &L.ev[e].lat_tab : nullptr;
        seeds = (T *)L.ev[e].seeds;
        S1 = S = L.ev[e].S;
        bx = lb;
    }
    const int64_t kb = BATCH ? 0 : blockIdx.y;
    if (refs) {
        const int64_t kr = kb < (int64_t)*n_refs ? kb : 0;
#pragma unroll
        for (int d = 0; d < 4; ++d) a.centre[d] = refs[kr * 4 + d];
    }
    int off[4];
    off[0] = 0;
    for (int d = 1; d < 4; ++d) off[d] = off[d - 1] + a.counts[d - 1];
    const int tot = off[3] + a.counts[3];
    const bool tab = !tp && tot <= kLatTab;
    if (tab) {
        for (int i = threadIdx.x; i < tot; i += blockDim.x) {
            const int d = i < off[1] ? 0 : (i < off[2] ? 1 : (i < off[3] ? 2 : 3));
            const int k = i - off[d];
            const double v = lattice_node(a.centre[d], a.half_width[d], a.counts[d], k);
            nodes[i] = v;
            if (d == 1) sincos(v, &sphi[k], &cphi[k]);
        }
        __syncthreads();
    }
    const int64_t s = bx * blockDim.x + threadIdx.x;
    if (s >= S1) return;
    int b[4];
    b[0] = a.counts[0] % 2 == 0 ? 2 : 1;
#pragma unroll
    for (int d = 1; d < 3; ++d) b[d] = a.counts[d] % 4 == 0 ? 4 : (a.counts[d] % 2 == 0 ? 2 : 1);
    b[3] = 1;
    const int64_t vol = (int64_t)b[0] * b[1] * b[2] * b[3];
    int64_t blk = s / vol, in = s % vol;
    int ii[4];
#pragma unroll
    for (int d = 3; d >= 0; --d) {
        const int nb = a.counts[d] / b[d];
        const int i_in = (int)(in % b[d]);
        in /= b[d];
        const int i_bl = (int)(blk % nb);
        blk /= nb;
        ii[d] = i_bl * b[d] + i_in;
    }
    double v[4], sp, cp;
    if (tp) {
#pragma unroll
        for (int d = 0; d < 4; ++d) v[d] = tp->node[off[d] + ii[d]];
        sp = tp->sphi[ii[1]];
        cp = tp->cphi[ii[1]];
    } else if (tab) {
#pragma unroll
        for (int d = 0; d < 4; ++d) v[d] = nodes[off[d] + ii[d]];
        sp = sphi[ii[1]];
        cp = cphi[ii[1]];
    } else {
#pragma unroll
        for (int d = 0; d < 4; ++d) v[d] = lattice_node(a.centre[d], a.half_width[d], a.counts[d], ii[d]);
        sincos(v[1], &sp, &cp);
    }
    const int64_t o = kb * S1 + s;
    seeds[0 * S + o] = (T)a.vx;
    seeds[1 * S + o] = (T)a.vy;
    seeds[2 * S + o] = (T)v[0];
    seeds[3 * S + o] = (T)__dmul_rn(v[3], cp);
    seeds[4 * S + o] = (T)__dmul_rn(v[3], sp);
    seeds[5 * S + o] = (T)v[2];
    if (a.charge_out) a.charge_out[o] = (int8_t)a.charge;
}

template <typename T>
__device__ __forceinline__ bool outside_region(T x, T y, T z, T zmin, T zmax, T rmax2)
{
    return z < zmin || z > zmax || x * x + y * y > rmax2;
}

// Map of one recording interval (stride RK4 steps) in a uniform axial field.  With P = px + i py
// and X = x + i y, one RK4 step is P' = m P, X' = X + n P, z' = z + dz (device.cuh), so `stride`
// steps are P' = m^k P, X' = X + n (m^k - 1) / (m - 1) P, z' = z + k dz: the same map in exact
// arithmetic, formed once per seed in double and then applied once per recorded state.  m^k - 1 is
// built by binary powering on A = m - 1 ((1 + A)(1 + B) - 1 = A + B + A B), never forming 1 + A,
// so nothing cancels.
__device__ __forceinline__ void axial_interval(double am1, double b, double c, double d, double dz,
                                               int k, double out[5])
{
    const double a0r = am1, a0i = -b;          // m - 1
    double Rr = 0.0, Ri = 0.0;                 // m^(bits taken so far) - 1
    double Br = a0r, Bi = a0i;                 // m^(2^j) - 1
    for (int e = k; e > 0; e >>= 1) {
        if (e & 1) {
            const double r = Rr + Br + (Rr * Br - Ri * Bi);
            const double i = Ri + Bi + (Rr * Bi + Ri * Br);
            Rr = r;
            Ri = i;
        }
        const double r = 2.0 * Br + (Br * Br - Bi * Bi);
        const double i = 2.0 * Bi + 2.0 * Br * Bi;
        Br = r;
        Bi = i;
    }
    // sum of m^j for j < k: (m^k - 1) / (m - 1), or k when the step does not turn
    double Sr = (double)k, Si = 0.0;
    const double den = a0r * a0r + a0i * a0i;
    if (den > 0.0) {
        const double inv = 1.0 / den;
        Sr = (Rr * a0r + Ri * a0i) * inv;
        Si = (Ri * a0r - Rr * a0i) * inv;
    }
    const double nr = c, ni = -d;              // n
    out[0] = Rr;                               // am1 of the interval
    out[1] = -Ri;                              // b
    out[2] = nr * Sr - ni * Si;                // c
    out[3] = -(nr * Si + ni * Sr);             // d
    out[4] = dz * k;                           // dz
}

// The same interval map for the FP32 kernel, in float-float arithmetic (device.cuh) from the
// seed's float momentum: P0 = |p| and the single-step coefficients, then the binary powering and
// the geometric sum, each carried to ~48 bits and rounded to float once at the end.
__device__ __forceinline__ AxialStep<float> axial_interval_ff(float px, float py, float pz, int q,
                                                              float bz, ff h, int k)
{
    auto sq = [](float v) {
        const float p = __fmul_rn(v, v);
        return ff{p, __fmaf_rn(v, v, -p)};
    };
    const ff P0 = ff_sqrt(ff_add(ff_add(sq(px), sq(py)), sq(pz)));
    const ff ip = ff_recip(P0);
    const ff w = ff_mulf(ff_mul(ff_of(kKappa), ip), (float)q * bz);
    const ff t = ff_mul(h, w);
    const ff t2 = ff_mul(t, t);
    const ff hp = ff_mul(h, ip);
    const float t2f = t2.hi;
    const ff g = ff_renorm(1.f, -t2f * (1.f / 6.f));                        // 1 - t^2/6
    const ff a0r = ff_mul(t2, ff_renorm(-0.5f, t2f * (1.f / 24.f)));       // am1
    const ff a0i = ff_neg(ff_mul(t, g));                                   // -b
    const ff c = ff_mul(hp, g);
    const ff d = ff_mul(ff_mul(hp, t), ff_renorm(0.5f, -t2f * (1.f / 24.f)));
    // m^k - 1 by binary powering on A = m - 1, as in axial_interval
    ff Rr{0.f, 0.f}, Ri{0.f, 0.f}, Br = a0r, Bi = a0i;
    bool first = true;
    for (int e = k; e > 0; e >>= 1) {
        if (e & 1) {
            if (first) {
                Rr = Br;
                Ri = Bi;
                first = false;
            } else {
                const ff r = ff_add(ff_add(Rr, Br), ff_sub(ff_mul(Rr, Br), ff_mul(Ri, Bi)));
                const ff i = ff_add(ff_add(Ri, Bi), ff_add(ff_mul(Rr, Bi), ff_mul(Ri, Br)));
                Rr = r;
                Ri = i;
            }
        }
        if (e > 1) {
            const ff r = ff_add(ff_mulf(Br, 2.f), ff_sub(ff_mul(Br, Br), ff_mul(Bi, Bi)));
            const ff i = ff_mulf(ff_add(Bi, ff_mul(Br, Bi)), 2.f);
            Br = r;
            Bi = i;
        }
    }
    // sum of m^j, j < k: (m^k - 1) / (m - 1), or k when the step does not turn
    ff Sr{(float)k, 0.f}, Si{0.f, 0.f};
    const ff den = ff_add(ff_mul(a0r, a0r), ff_mul(a0i, a0i));
    if (den.hi > 0.f) {
        const ff inv = ff_recip(den);
        Sr = ff_mul(ff_add(ff_mul(Rr, a0r), ff_mul(Ri, a0i)), inv);
        Si = ff_mul(ff_sub(ff_mul(Ri, a0r), ff_mul(Rr, a0i)), inv);
    }
    AxialStep<float> ks;
    ks.am1 = Rr.hi;
    ks.b = -Ri.hi;
    ks.c = ff_add(ff_mul(c, Sr), ff_mul(d, Si)).hi;
    ks.d = ff_sub(ff_mul(d, Sr), ff_mul(c, Si)).hi;
    ks.dz = ff_mulf(ff_mulf(hp, pz), (float)k).hi;
    return ks;
}

// One recording interval (stride RK4 steps) of one seed.  In an axial field the interval's map is
// applied once (axial_interval); FP32 adds its increments to the compensated (hi, lo) state.  pz
// is constant in an axial field.  Other fields take the steps one by one.  STRIDE > 0 fixes the
// number of steps at compile time; 0 takes a.stride.
template <typename T, class F, int STRIDE>
__device__ __forceinline__ void advance_interval(const F &f, const PropArgs &a, const AxialStep<T> &ks,
                                                 T c, T ip, T h, T y[6], float lo[6],
                                                 typename F::Cell &cell)
{
    const int stride = STRIDE > 0 ? STRIDE : a.stride;
    if constexpr (sizeof(T) == 4 && F::kAxial) {
        const float px = y[3], py = y[4];
        fast_two_sum_add(y[0], lo[0], ks.c * px + ks.d * py);
        fast_two_sum_add(y[1], lo[1], ks.c * py - ks.d * px);
        fast_two_sum_add(y[2], lo[2], ks.dz);
        fast_two_sum_add(y[3], lo[3], ks.am1 * px + ks.b * py);
        fast_two_sum_add(y[4], lo[4], ks.am1 * py - ks.b * px);
    } else if constexpr (F::kAxial) {
        T inc[6];
        axial_increment<T>(ks, y, inc);
#pragma unroll
        for (int i = 0; i < 6; ++i) y[i] += inc[i];
    } else if constexpr (sizeof(T) == 4) {
        for (int st = 0; st < stride; ++st) {
            float inc[6];
            rk4_increment_cell<float, F>(f, cell, c, ip, y, h, inc);
#pragma unroll
            for (int i = 0; i < 6; ++i) two_sum_add(y[i], lo[i], inc[i]);
        }
    } else {
        for (int st = 0; st < stride; ++st) {
            T inc[6];
            rk4_increment_cell<T, F>(f, cell, c, ip, y, h, inc);
#pragma unroll
            for (int i = 0; i < 6; ++i) y[i] += inc[i];
        }
    }
}

// BATCH: one launch for a batch of events; block b belongs to the event that batch_find gives.
template <typename T, class F, int STRIDE, bool BATCH>
__global__ void __launch_bounds__(128) propagate_kernel(F f, PropArgs a, BatchLaunch L)
{
    int64_t bx = blockIdx.x;
    if constexpr (BATCH) {
        int e;
        int64_t lb;
        if (!batch_find(L.prop_start, L.B, blockIdx.x, e, lb)) return;
        a = L.ev[e].prop;
        bx = lb;
    }
    const int64_t s = bx * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31;
    const bool valid = s < a.S;
    const bool wb = a.bounds != nullptr;   // whole warps then stay in the loop (warp reductions)
    if (!valid && !wb) return;
    // a warp with no seed at all (past the end) has no bounds entry: it leaves as a whole
    if ((s & ~(int64_t)31) >= a.S) return;
    const int64_t S = a.S;
    const T *__restrict__ seeds = (const T *)a.seeds;
    T *__restrict__ pts = (T *)a.points;
    const int64_t plane = (int64_t)a.n_rec * S;
    const int n_rec = a.n_rec;

    T y[6] = {T(0), T(0), T(0), T(0), T(0), T(0)};
    int q = 0;
    if (valid) {
#pragma unroll
        for (int c = 0; c < 6; ++c) y[c] = seeds[c * S + s];
        q = a.charge[s];
    }
    constexpr bool kFF = sizeof(T) == 4 && F::kAxial;   // FP32 axial: no double arithmetic at all
    T c = T(0), ip = T(0);
    double ipd = 1.0;
    if constexpr (!kFF) {
        const double pd = valid ? sqrt((double)y[3] * y[3] + (double)y[4] * y[4] + (double)y[5] * y[5]) : 1.0;
        ipd = 1.0 / pd;
        c = (T)(kKappa * q * ipd);
        ip = (T)ipd;
    }
    const T h = kFF ? (T)a.h_ff.hi : (T)a.h;
    const T zmin = kFF ? (T)a.lim_f[0] : (T)a.zmin, zmax = kFF ? (T)a.lim_f[1] : (T)a.zmax;
    const T rmax2 = kFF ? (T)a.lim_f[2] : (T)(a.rmax * a.rmax);
    const T R0 = kFF ? (T)a.lim_f[3] : (T)a.R0, R1 = kFF ? (T)a.lim_f[4] : (T)a.R1;
    // uniform axial field: the interval's map is fixed per seed
    AxialStep<T> ks{};
    if constexpr (kFF) {
        ks = axial_interval_ff(y[3], y[4], y[5], valid ? q : 0, f.bz, a.h_ff,
                               STRIDE > 0 ? STRIDE : a.stride);
    } else if constexpr (F::kAxial) {
        const double w = kKappa * q * (double)f.bz * ipd;
        const double t = a.h * w, t2 = t * t, hp = a.h * ipd;
        double m[5];
        axial_interval(t2 * (-0.5 + t2 / 24.0), t * (1.0 - t2 / 6.0), hp * (1.0 - t2 / 6.0),
                       hp * t * (0.5 - t2 / 24.0), hp * (double)y[5], STRIDE > 0 ? STRIDE : a.stride, m);
        ks.am1 = (T)m[0];
        ks.b = (T)m[1];
        ks.c = (T)m[2];
        ks.d = (T)m[3];
        ks.dz = (T)m[4];
    }
    float lo[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};   // FP32: low words of the compensated state
    typename F::Cell cell;                          // tabulated field: the cell of the last lookup

    // Bounding spheres of the segments whose centre is the state just recorded (see device.cuh);
    // lanes that stopped earlier contribute their last recorded state if the segment holds it.
    // The next centres are tracked incrementally.
    float4 *tab = wb ? (float4 *)a.bounds + (s >> 5) * kBoundsPerGroup : nullptr;
    int last_k = 0;
    const int G0 = a.G0, G1 = a.G1;
    int j1 = 0, m1 = 0, st1 = 0, se1 = min(G0, n_rec);   // current level-1 segment
    int c1 = segment_centre(0, G1, se1);
    int j0 = 0, sb0 = 0;                                 // current super-segment
    int c0 = segment_centre(0, G0, se1);

    if (wb) {
        for (int i = lane; i < kBoundsPerGroup; i += 32) tab[i] = make_float4(0.f, 0.f, 0.f, -1.f);
        __syncwarp();
    }
    if (valid) {
#pragma unroll
        for (int cc = 0; cc < 6; ++cc) pts[cc * plane + s] = y[cc];
    }
    int n = 1;
    bool active = valid && !outside_region<T>(y[0], y[1], y[2], zmin, zmax, rmax2);
    for (int r = 0; r < n_rec; ++r) {
        if (r > 0 && active) {
            advance_interval<T, F, STRIDE>(f, a, ks, c, ip, h, y, lo, cell);
            const int64_t o = (int64_t)r * S + s;
#pragma unroll
            for (int cc = 0; cc < 6; ++cc) pts[cc * plane + o] = y[cc];
            n = r + 1;
            last_k = r;
            if (outside_region<T>(y[0], y[1], y[2], zmin, zmax, rmax2)) active = false;
        }
        if (wb) {
            if (G1 == 1) {
                // every recorded state is a level-1 segment of its own: (j1, m1) = (r / G0, r % G0)
                const float4 sp = warp_sphere<T>(valid && last_k >= r, y[0], y[1], y[2], R1);
                if (lane == 0) tab[kN0Max + j1 * kN1Max + m1] = sp;
                if (++m1 == G0) {
                    m1 = 0;
                    ++j1;
                }
            } else if (r == c1) {
                const float4 sp = warp_sphere<T>(valid && last_k >= st1, y[0], y[1], y[2], R1);
                if (lane == 0) tab[kN0Max + j1 * kN1Max + m1] = sp;
                ++m1;
                st1 += G1;
                if (st1 >= se1) {
                    ++j1;
                    m1 = 0;
                    st1 = j1 * G0;
                    se1 = min(st1 + G0, n_rec);
                }
                c1 = st1 < n_rec ? segment_centre(st1, G1, se1) : 0x7fffffff;
            }
            if (r == c0) {
                const float4 sp = warp_sphere<T>(valid && last_k >= sb0, y[0], y[1], y[2], R0);
                if (lane == 0) tab[j0] = sp;
                ++j0;
                sb0 += G0;
                c0 = sb0 < n_rec ? segment_centre(sb0, G0, min(sb0 + G0, n_rec)) : 0x7fffffff;
            }
        } else if (!active) {
            break;
        }
    }
    if (valid) a.n_valid[s] = n;
}

// Few seeds, uniform axial field, FP64: one warp per (32-seed group, super-segment).  A track's
// recorded states are the powers of one interval map (see axial_interval), so each super-segment
// [r0, r1) starts from the seed mapped over r0 intervals at once and then steps interval by
// interval as propagate_kernel does: with 4,096 seeds the sequential kernel has one warp per SM,
// one of its four schedulers issuing FP64 work; here each group has one warp per super-segment
// (up to 8).  The states are those of the sequential recording up to rounding (the map of r0
// intervals against r0 applications of the one-interval map).  n_valid: the caller's array is set
// to a large value first (a byte memset), then each block lowers it to its first state outside the
// target region plus one, and the last block to n_rec.  Spheres: a lane whose track left the region
// in an earlier block still contributes its (extrapolated) states, which only makes the sphere
// larger; within the block a lane stops contributing to segments after its exit, as in
// propagate_kernel.
template <int STRIDE>
__global__ void __launch_bounds__(32) propagate_blocks_kernel(FieldAxial<double> f, PropArgs a)
{
    const int n_rec = a.n_rec, G0 = a.G0, G1 = a.G1;
    const int n0 = (n_rec + G0 - 1) / G0;
    const int64_t g = blockIdx.x / n0;
    const int j = (int)(blockIdx.x % n0);
    const int lane = threadIdx.x;
    const int64_t S = a.S;
    const int64_t s = g * 32 + lane;
    const bool valid = s < S;
    const double *__restrict__ seeds = (const double *)a.seeds;
    double *__restrict__ pts = (double *)a.points;
    const int64_t plane = (int64_t)n_rec * S;

    double y[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    int q = 0;
    if (valid) {
#pragma unroll
        for (int c = 0; c < 6; ++c) y[c] = seeds[c * S + s];
        q = a.charge[s];
    }
    // the one-step coefficients and the interval map exactly as propagate_kernel forms them
    const double pd = valid ? sqrt((double)y[3] * y[3] + (double)y[4] * y[4] + (double)y[5] * y[5]) : 1.0;
    const double ipd = 1.0 / pd;
    const double w = kKappa * q * (double)f.bz * ipd;
    const double t = a.h * w, t2 = t * t, hp = a.h * ipd;
    const double s_am1 = t2 * (-0.5 + t2 / 24.0), s_b = t * (1.0 - t2 / 6.0), s_c = hp * (1.0 - t2 / 6.0),
                 s_d = hp * t * (0.5 - t2 / 24.0), s_dz = hp * (double)y[5];
    const int stride = STRIDE > 0 ? STRIDE : a.stride;
    double m[5];
    axial_interval(s_am1, s_b, s_c, s_d, s_dz, stride, m);
    const AxialStep<double> ks{m[0], m[1], m[2], m[3], m[4]};
    const int r0 = j * G0, r1 = min(r0 + G0, n_rec);
    if (r0 > 0) {
        // the state after r0 intervals: the map of r0 * stride steps applied once
        axial_interval(s_am1, s_b, s_c, s_d, s_dz, r0 * stride, m);
        const AxialStep<double> k0{m[0], m[1], m[2], m[3], m[4]};
        double inc[6];
        axial_increment<double>(k0, y, inc);
#pragma unroll
        for (int i = 0; i < 6; ++i) y[i] += inc[i];
    }

    const double zmin = a.zmin, zmax = a.zmax, rmax2 = a.rmax * a.rmax;
    // A lane whose states in [r0, r1) provably stay inside the target region skips the per-state
    // test: in this field the track is a circle of radius R = pT / |P0 w| about
    // C = (x, y) + (py, -px) / (P0 w) (in the transverse plane) and z moves by ks.dz per interval,
    // so all its states lie within |C| + R of the axis and between the z of the first and the last
    // state.  The 1 um margin is far above the RK4 map's drift from that circle (~1e-13 m per turn)
    // and the rounding; lanes near the boundary keep the per-state test.
    bool safe = false;
    if (valid && w != 0.0) {
        const double pw = pd * w;
        const double cx = y[0] + y[4] / pw, cy = y[1] - y[3] / pw;
        const double rr = sqrt(y[3] * y[3] + y[4] * y[4]) / fabs(pw);
        const double rout = sqrt(cx * cx + cy * cy) + rr + 1e-6;
        const double z_end = y[2] + (double)(r1 - 1 - r0) * ks.dz;
        const double zlo = fmin(y[2], z_end) - 1e-6, zhi = fmax(y[2], z_end) + 1e-6;
        safe = rout * rout < rmax2 && zlo > zmin && zhi < zmax;
    }
    const bool wb = a.bounds != nullptr;
    float4 *tab = wb ? (float4 *)a.bounds + g * kBoundsPerGroup : nullptr;
    const int N1 = (r1 - r0 + G1 - 1) / G1;   // level-1 segments of this super-segment
    if (wb) {
        // entries no segment of this block fills; block 0 also clears the unused super-segments
        for (int mm = N1 + lane; mm < kN1Max; mm += 32)
            tab[kN0Max + j * kN1Max + mm] = make_float4(0.f, 0.f, 0.f, -1.f);
        if (j == 0)
            for (int i = lane; i < (kN0Max - n0) * (kN1Max + 1); i += 32) {
                const int jj = n0 + i / (kN1Max + 1), mm = i % (kN1Max + 1);
                if (mm == kN1Max)
                    tab[jj] = make_float4(0.f, 0.f, 0.f, -1.f);
                else
                    tab[kN0Max + jj * kN1Max + mm] = make_float4(0.f, 0.f, 0.f, -1.f);
            }
    }
    int exit_k = 0x7fffffff;                  // this lane's first state outside the region
    int m1 = 0, st1 = r0;
    int c1 = segment_centre(r0, G1, r1);
    const int c0 = segment_centre(r0, G0, r1);
    for (int r = r0; r < r1; ++r) {
        if (r > r0) {
            double inc[6];
            axial_increment<double>(ks, y, inc);
#pragma unroll
            for (int i = 0; i < 6; ++i) y[i] += inc[i];
        }
        if (valid) {
            const int64_t o = (int64_t)r * S + s;
#pragma unroll
            for (int cc = 0; cc < 6; ++cc) pts[cc * plane + o] = y[cc];
            if (!safe && exit_k == 0x7fffffff &&
                outside_region<double>(y[0], y[1], y[2], zmin, zmax, rmax2))
                exit_k = r;
        }
        if (wb) {
            if (r == c1) {
                const float4 sp = warp_sphere<double>(valid && exit_k >= st1, y[0], y[1], y[2], a.R1);
                if (lane == 0) tab[kN0Max + j * kN1Max + m1] = sp;
                ++m1;
                st1 += G1;
                c1 = st1 < r1 ? segment_centre(st1, G1, r1) : 0x7fffffff;
            }
            if (r == c0) {
                const float4 sp = warp_sphere<double>(valid, y[0], y[1], y[2], a.R0);
                if (lane == 0) tab[j] = sp;
            }
        }
    }
    if (valid) {
        if (exit_k != 0x7fffffff) atomicMin(a.n_valid + s, exit_k + 1);
        if (j == n0 - 1) atomicMin(a.n_valid + s, n_rec);
    }
}

static cudaError_t lattice_launch(comet_dtype dt, const LatArgs &a, const LatTable &t,
                                  const double *refs, const int32_t *n_refs, int K, void *seeds,
                                  int64_t S, cudaStream_t st)
{
    const int nt = 256;
    const int64_t S1 = S / K;
    const dim3 grid((unsigned)((S1 + nt - 1) / nt), (unsigned)K);
    const BatchLaunch none{};
    if (dt == COMET_F32)
        lattice_kernel<float, false><<<grid, nt, 0, st>>>(a, t, refs, n_refs, (float *)seeds, S1, S, none);
    else
        lattice_kernel<double, false><<<grid, nt, 0, st>>>(a, t, refs, n_refs, (double *)seeds, S1, S, none);
    return cudaGetLastError();
}

cudaError_t launch_lattice(comet_dtype dt, const LatArgs &a, const LatTable &t, void *seeds, int64_t S,
                           cudaStream_t st)
{
    return lattice_launch(dt, a, t, nullptr, nullptr, 1, seeds, S, st);
}

cudaError_t launch_lattice_refined(comet_dtype dt, const LatArgs &a, const double *refs,
                                   const int32_t *n_refs, int K, void *seeds, int64_t S,
                                   cudaStream_t st)
{
    // the centres are the references on the device: tabulated per block
    LatTable none;
    none.use = 0;
    return lattice_launch(dt, a, none, refs, n_refs, K, seeds, S, st);
}

cudaError_t launch_lattice_batch(comet_dtype dt, const BatchLaunch &L, cudaStream_t st)
{
    if (L.lat_blocks == 0) return cudaSuccess;
    const LatArgs none{};
    LatTable no_tab;
    no_tab.use = 0;
    if (dt == COMET_F32)
        lattice_kernel<float, true><<<L.lat_blocks, 256, 0, st>>>(none, no_tab, nullptr, nullptr, nullptr, 0, 0, L);
    else
        lattice_kernel<double, true><<<L.lat_blocks, 256, 0, st>>>(none, no_tab, nullptr, nullptr, nullptr, 0, 0, L);
    return cudaGetLastError();
}

template <typename T, class F, bool BATCH>
static void prop_launch(const F &fld, const PropArgs &a, int stride, unsigned nb, const BatchLaunch &L,
                        cudaStream_t st, int nt = 128)
{
    switch (stride) {
    case 1: propagate_kernel<T, F, 1, BATCH><<<nb, nt, 0, st>>>(fld, a, L); break;
    case 2: propagate_kernel<T, F, 2, BATCH><<<nb, nt, 0, st>>>(fld, a, L); break;
    case 4: propagate_kernel<T, F, 4, BATCH><<<nb, nt, 0, st>>>(fld, a, L); break;
    case 8: propagate_kernel<T, F, 8, BATCH><<<nb, nt, 0, st>>>(fld, a, L); break;
    default: propagate_kernel<T, F, 0, BATCH><<<nb, nt, 0, st>>>(fld, a, L); break;
    }
}

template <typename T, bool BATCH>
static void prop_dispatch(const comet_field &f, const PropArgs &a, int stride, unsigned nb,
                          const BatchLaunch &L, cudaStream_t st, int nt = 128)
{
    switch (field_kind(f)) {
    case FieldKind::Axial:
        prop_launch<T, FieldAxial<T>, BATCH>(FieldAxial<T>{(T)f.b[2]}, a, stride, nb, L, st, nt);
        break;
    case FieldKind::Uniform:
        prop_launch<T, FieldUniform<T>, BATCH>(FieldUniform<T>{(T)f.b[0], (T)f.b[1], (T)f.b[2]}, a,
                                               stride, nb, L, st, nt);
        break;
    case FieldKind::Table:
        prop_launch<T, FieldTable<T>, BATCH>(make_table<T>(f),
                                             a, stride, nb, L, st, nt);
        break;
    }
}

cudaError_t launch_propagate(comet_dtype dt, const comet_field &f, const PropArgs &a, bool blocks,
                             cudaStream_t st)
{
    // FP64 in a uniform axial field with fewer than four 32-seed groups per SM (when the context
    // allows it): one warp per (group, super-segment), each started from the composed interval map
    const int64_t groups = (a.S + 31) / 32;
    const int n0 = a.G0 > 0 ? (a.n_rec + a.G0 - 1) / a.G0 : 1;
    if (blocks && dt == COMET_F64 && field_kind(f) == FieldKind::Axial && n0 > 1 &&
        groups < (int64_t)device_sm_count() * 4) {
        cudaError_t e = cudaMemsetAsync(a.n_valid, 0x7f, (size_t)a.S * sizeof(int32_t), st);
        if (e != cudaSuccess) return e;
        const unsigned nb = (unsigned)(groups * n0);
        const FieldAxial<double> fa{f.b[2]};
        switch (a.stride) {
        case 1: propagate_blocks_kernel<1><<<nb, 32, 0, st>>>(fa, a); break;
        case 2: propagate_blocks_kernel<2><<<nb, 32, 0, st>>>(fa, a); break;
        case 4: propagate_blocks_kernel<4><<<nb, 32, 0, st>>>(fa, a); break;
        case 8: propagate_blocks_kernel<8><<<nb, 32, 0, st>>>(fa, a); break;
        default: propagate_blocks_kernel<0><<<nb, 32, 0, st>>>(fa, a); break;
        }
        return cudaGetLastError();
    }
    // one seed per thread; with fewer seeds than 128 per SM, one warp per CTA, so that the seeds
    // spread over as many SMs as possible (the search bounds are per warp either way)
    const int nt = a.S < (int64_t)device_sm_count() * 128 ? 32 : 128;
    const unsigned nb = (unsigned)((a.S + nt - 1) / nt);
    const BatchLaunch none{};
    if (dt == COMET_F32)
        prop_dispatch<float, false>(f, a, a.stride, nb, none, st, nt);
    else
        prop_dispatch<double, false>(f, a, a.stride, nb, none, st, nt);
    return cudaGetLastError();
}

cudaError_t launch_propagate_batch(comet_dtype dt, const comet_field &f, int stride, const BatchLaunch &L,
                                   cudaStream_t st)
{
    if (L.prop_blocks == 0) return cudaSuccess;
    const PropArgs none{};
    if (dt == COMET_F32)
        prop_dispatch<float, true>(f, none, stride, L.prop_blocks, L, st);
    else
        prop_dispatch<double, true>(f, none, stride, L.prop_blocks, L, st);
    return cudaGetLastError();
}

} // namespace comet
