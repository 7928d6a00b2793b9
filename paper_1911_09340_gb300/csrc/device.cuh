// Device building blocks of the seed scan (sm_103a): field evaluation, RK4 on y = (x, p), the
// compensated FP32 state update, the point-to-wire distance, the virtual-plane DCA refinement and
// the shared-memory staging of small arrays with the bulk-copy (TMA) engine.
//
// Equations of motion (arc length s, P0 = |p| of the seed, KAPPA = 299.792458 MeV/c per (T m)):
//     dx/ds = p / P0,    dp/ds = (KAPPA q / P0) p x B(x).
// In a uniform field this is the helix of Sec. 1; the paper integrates it with an RKN method
// (Sec. 2.1), the scan here with classic fixed-step RK4.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.h"   // struct ff

namespace comet {

constexpr double kKappa = 299.792458;

// ------------------------------------------------------------------------------------------------
// Fields
// ------------------------------------------------------------------------------------------------

// Uniform field along z: B = (0, 0, bz).  dp/ds reduces to w (py, -px, 0) with w = c bz.
template <typename T>
struct FieldAxial {
    static constexpr bool kAxial = true;
    T bz;
    __device__ __forceinline__ void at(T, T, T, T &bx, T &by, T &bz_) const
    {
        bx = T(0);
        by = T(0);
        bz_ = bz;
    }
    struct Cell {};
    __device__ __forceinline__ void at_cell(Cell &, T x, T y, T z, T &bx, T &by, T &bz_) const
    {
        at(x, y, z, bx, by, bz_);
    }
    __device__ __forceinline__ void at_enter(Cell &, T x, T y, T z, T &bx, T &by, T &bz_) const
    {
        at(x, y, z, bx, by, bz_);
    }
};

// Uniform field of any direction.
template <typename T>
struct FieldUniform {
    static constexpr bool kAxial = false;
    T b0, b1, b2;
    __device__ __forceinline__ void at(T, T, T, T &bx, T &by, T &bz) const
    {
        bx = b0;
        by = b1;
        bz = b2;
    }
    struct Cell {};
    __device__ __forceinline__ void at_cell(Cell &, T x, T y, T z, T &bx, T &by, T &bz_) const
    {
        at(x, y, z, bx, by, bz_);
    }
    __device__ __forceinline__ void at_enter(Cell &, T x, T y, T z, T &bx, T &by, T &bz_) const
    {
        at(x, y, z, bx, by, bz_);
    }
};

// Trilinear interpolation of a float32 table [3][nz][ny][nx]; coordinates clamped to the grid.
template <typename T>
struct FieldTable {
    static constexpr bool kAxial = false;
    const float *__restrict__ tab;
    int nx, ny, nz;
    T ox, oy, oz, inv_sp;
    int il;   // layout: 0 = [3][nz][ny][nx], 1 = [nz][ny][nx][4] (one 16-byte load per node)

    __device__ __forceinline__ static void cell(T g, int n, int &i, T &t)
    {
        g = g < T(0) ? T(0) : g;
        g = g > T(n - 1) ? T(n - 1) : g;
        T fl = floor(g);
        i = (int)fl;
        i = i > n - 2 ? n - 2 : i;
        t = g - T(i);
    }

    // The eight corner nodes of the grid cell a lane used last (base: index of its node 000; none
    // at first).  Lookups in the same cell take them from registers: the RK4 stages 2 and 3 of a
    // step are microns apart, and so are stage 4 and the next step's stage 1, so about half of the
    // recording's lookups need no node load.  The interpolation is the same arithmetic on the same
    // node values as at(), so results are bit-identical.
    struct Cell {
        int64_t base = -1;
        T fx = T(-1e30), fy = T(-1e30), fz = T(-1e30);   // its node 000 in grid units
        // per x edge e = (z bit, y bit) and component c: the node at x = 0 and the difference to
        // the node at x = 1, both as the interpolation rounds them
        T v0[4][3], dx[4][3];
    };

    __device__ __forceinline__ static T lerp3(const Cell &cc, int c, T tx, T ty, T tz)
    {
        const T a00 = cc.v0[0][c] + tx * cc.dx[0][c];
        const T a01 = cc.v0[1][c] + tx * cc.dx[1][c];
        const T a10 = cc.v0[2][c] + tx * cc.dx[2][c];
        const T a11 = cc.v0[3][c] + tx * cc.dx[3][c];
        const T b0 = a00 + ty * (a01 - a00);
        const T b1 = a10 + ty * (a11 - a10);
        return b0 + tz * (b1 - b0);
    }

    __device__ __forceinline__ void at_cell(Cell &cc, T x, T y, T z, T &bx, T &by, T &bz) const
    {
        const T gx = (x - ox) * inv_sp, gy = (y - oy) * inv_sp, gz = (z - oz) * inv_sp;
        // inside the cached cell, 0 <= g - i < 1 in every dimension: g needs no clamping there,
        // floor(g) = i, and g - i is exact (Sterbenz), so these are the fractions cell() gives
        T tx = gx - cc.fx, ty = gy - cc.fy, tz = gz - cc.fz;
        if (!(tx >= T(0) && tx < T(1) && ty >= T(0) && ty < T(1) && tz >= T(0) && tz < T(1)))
            enter(cc, gx, gy, gz, tx, ty, tz);
        bx = lerp3(cc, 0, tx, ty, tz);
        by = lerp3(cc, 1, tx, ty, tz);
        bz = lerp3(cc, 2, tx, ty, tz);
    }

    // The lookup through enter() without the in-cell test (for a lookup that has probably moved).
    __device__ __forceinline__ void at_enter(Cell &cc, T x, T y, T z, T &bx, T &by, T &bz) const
    {
        T tx, ty, tz;
        enter(cc, (x - ox) * inv_sp, (y - oy) * inv_sp, (z - oz) * inv_sp, tx, ty, tz);
        bx = lerp3(cc, 0, tx, ty, tz);
        by = lerp3(cc, 1, tx, ty, tz);
        bz = lerp3(cc, 2, tx, ty, tz);
    }

    // A lookup outside the cached cell: the cell of (gx, gy, gz) as at() finds it, its fractions,
    // and its corner nodes unless it is the cached one after all (clamped at the grid's edges).
    __device__ __forceinline__ void enter(Cell &cc, T gx, T gy, T gz, T &tx, T &ty, T &tz) const
    {
        int ix, iy, iz;
        cell(gx, nx, ix, tx);
        cell(gy, ny, iy, ty);
        cell(gz, nz, iz, tz);
        cc.fx = T(ix);
        cc.fy = T(iy);
        cc.fz = T(iz);
        const int64_t base = ((int64_t)iz * ny + iy) * nx + ix;
        if (base != cc.base) {
            cc.base = base;
            const int64_t sy = nx, sz = (int64_t)nx * ny;
            // corner j = (z bit, y bit, x bit), x fastest
            const int64_t off[8] = {0, 1, sy, sy + 1, sz, sz + 1, sz + sy, sz + sy + 1};
            float v[8][3];
            if (il) {
                const float4 *q = (const float4 *)tab + base;
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const float4 n = __ldg(q + off[j]);
                    v[j][0] = n.x;
                    v[j][1] = n.y;
                    v[j][2] = n.z;
                }
            } else {
                const int64_t plane = (int64_t)nz * ny * nx;
#pragma unroll
                for (int c = 0; c < 3; ++c)
#pragma unroll
                    for (int j = 0; j < 8; ++j) v[j][c] = __ldg(tab + c * plane + base + off[j]);
            }
#pragma unroll
            for (int e = 0; e < 4; ++e)
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    cc.v0[e][c] = (T)v[2 * e][c];
                    cc.dx[e][c] = (T)v[2 * e + 1][c] - (T)v[2 * e][c];
                }
        }
    }

    __device__ __forceinline__ void at(T x, T y, T z, T &bx, T &by, T &bz) const
    {
        int ix, iy, iz;
        T tx, ty, tz;
        cell((x - ox) * inv_sp, nx, ix, tx);
        cell((y - oy) * inv_sp, ny, iy, ty);
        cell((z - oz) * inv_sp, nz, iz, tz);
        const size_t plane = (size_t)nz * ny * nx;
        const size_t base = ((size_t)iz * ny + iy) * nx + ix;
        const size_t sy = (size_t)nx, sz = (size_t)nx * ny;
        T out[3];
        if (il) {
            const float4 *q = (const float4 *)tab + base;
            const float4 n000 = __ldg(q), n001 = __ldg(q + 1), n010 = __ldg(q + sy), n011 = __ldg(q + sy + 1);
            const float4 n100 = __ldg(q + sz), n101 = __ldg(q + sz + 1), n110 = __ldg(q + sz + sy),
                         n111 = __ldg(q + sz + sy + 1);
            auto lerp3 = [&](float v000, float v001, float v010, float v011, float v100, float v101,
                             float v110, float v111) {
                const T a00 = (T)v000 + tx * ((T)v001 - (T)v000);
                const T a01 = (T)v010 + tx * ((T)v011 - (T)v010);
                const T a10 = (T)v100 + tx * ((T)v101 - (T)v100);
                const T a11 = (T)v110 + tx * ((T)v111 - (T)v110);
                const T b0 = a00 + ty * (a01 - a00);
                const T b1 = a10 + ty * (a11 - a10);
                return b0 + tz * (b1 - b0);
            };
            bx = lerp3(n000.x, n001.x, n010.x, n011.x, n100.x, n101.x, n110.x, n111.x);
            by = lerp3(n000.y, n001.y, n010.y, n011.y, n100.y, n101.y, n110.y, n111.y);
            bz = lerp3(n000.z, n001.z, n010.z, n011.z, n100.z, n101.z, n110.z, n111.z);
            return;
        }
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const float *p = tab + c * plane + base;
            T v000 = (T)__ldg(p), v001 = (T)__ldg(p + 1);
            T v010 = (T)__ldg(p + sy), v011 = (T)__ldg(p + sy + 1);
            T v100 = (T)__ldg(p + sz), v101 = (T)__ldg(p + sz + 1);
            T v110 = (T)__ldg(p + sz + sy), v111 = (T)__ldg(p + sz + sy + 1);
            T a00 = v000 + tx * (v001 - v000);
            T a01 = v010 + tx * (v011 - v010);
            T a10 = v100 + tx * (v101 - v100);
            T a11 = v110 + tx * (v111 - v110);
            T b0 = a00 + ty * (a01 - a00);
            T b1 = a10 + ty * (a11 - a10);
            out[c] = b0 + tz * (b1 - b0);
        }
        bx = out[0];
        by = out[1];
        bz = out[2];
    }
};

template <typename T>
inline FieldTable<T> make_table(const comet_field &f)
{
    return FieldTable<T>{(const float *)f.table, f.nx, f.ny, f.nz, (T)f.origin[0], (T)f.origin[1],
                         (T)f.origin[2], (T)(1.0 / f.spacing), f.kind == 2 ? 1 : 0};
}

// ------------------------------------------------------------------------------------------------
// RK4
// ------------------------------------------------------------------------------------------------

// Uniform axial field, B = (0, 0, Bz): with w = KAPPA q Bz / P0 the ODE is linear,
// dx/ds = p / P0, d(px, py)/ds = w (py, -px), and one classic RK4 step of length h is exactly the map
//     dp  = (A - 1) p + B Jp,          A - 1 = -t^2/2 + t^4/24,   B = t - t^3/6,
//     dxy = C p + D Jp,                C = (h/P0)(1 - t^2/6),     D = (h/P0)(t/2 - t^3/24),
//     dz  = h pz / P0,                 t = h w,  Jp = (py, -px),
// i.e. the sums k1 + 2 k2 + 2 k3 + k4 of the four stages collected into powers of t (J^2 = -1).  Same
// step as the staged form in exact arithmetic, with about a fifth of the operations.
template <typename T>
struct AxialStep {
    T am1, b, c, d, dz;
};

template <typename T>
__device__ __forceinline__ AxialStep<T> axial_step_coeffs(T w, T ip, T pz, T h)
{
    const T t = h * w, t2 = t * t;
    const T hp = h * ip;
    AxialStep<T> k;
    k.am1 = t2 * (T(-0.5) + t2 * T(1.0 / 24.0));
    k.b = t * (T(1) - t2 * T(1.0 / 6.0));
    k.c = hp * (T(1) - t2 * T(1.0 / 6.0));
    k.d = hp * t * (T(0.5) - t2 * T(1.0 / 24.0));
    k.dz = hp * pz;
    return k;
}

template <typename T>
__device__ __forceinline__ void axial_increment(const AxialStep<T> &k, const T y[6], T inc[6])
{
    inc[0] = k.c * y[3] + k.d * y[4];
    inc[1] = k.c * y[4] - k.d * y[3];
    inc[2] = k.dz;
    inc[3] = k.am1 * y[3] + k.b * y[4];
    inc[4] = k.am1 * y[4] - k.b * y[3];
    inc[5] = T(0);
}

// The four stages of one classic RK4 step of length h from state y, the field from look(x, y, z,
// bx, by, bz): inc = h/6 (k1 + 2 k2 + 2 k3 + k4).  c = KAPPA q / P0, ip = 1 / P0.
template <typename T, class Look>
__device__ __forceinline__ void rk4_stages(Look look, T c, T ip, const T y[6], T h, T inc[6])
{
    const T hh = T(0.5) * h;
    const T h6 = h / T(6);
    T k[4][6];
    T t[6];
#pragma unroll
    for (int i = 0; i < 6; ++i) t[i] = y[i];
#pragma unroll
    for (int st = 0; st < 4; ++st) {
        T bx, by, bz;
        look(st, t[0], t[1], t[2], bx, by, bz);
        k[st][0] = t[3] * ip;
        k[st][1] = t[4] * ip;
        k[st][2] = t[5] * ip;
        k[st][3] = c * (t[4] * bz - t[5] * by);
        k[st][4] = c * (t[5] * bx - t[3] * bz);
        k[st][5] = c * (t[3] * by - t[4] * bx);
        if (st < 3) {
            const T a = st < 2 ? hh : h;
#pragma unroll
            for (int i = 0; i < 6; ++i) t[i] = y[i] + a * k[st][i];
        }
    }
#pragma unroll
    for (int i = 0; i < 6; ++i)
        inc[i] = h6 * ((k[0][i] + T(2) * (k[1][i] + k[2][i])) + k[3][i]);
}

// Increment of one classic RK4 step of length h from state y: inc = h/6 (k1 + 2 k2 + 2 k3 + k4).
// c = KAPPA q / P0, ip = 1 / P0.
template <typename T, class F>
__device__ __forceinline__ void rk4_increment(const F &f, T c, T ip, const T y[6], T h, T inc[6])
{
    if constexpr (F::kAxial) {
        axial_increment<T>(axial_step_coeffs<T>(c * f.bz, ip, y[5], h), y, inc);
    } else {
        rk4_stages<T>([&](int, T x0, T x1, T x2, T &bx, T &by, T &bz) { f.at(x0, x1, x2, bx, by, bz); },
                      c, ip, y, h, inc);
    }
}

// The same step with the lane's field cell carried from lookup to lookup (F::at_cell): for the
// recording, whose consecutive lookups mostly fall in the cell of the one before.  Stages 1 and 3
// lie microns from the lookup before them and test the cached cell; stages 2 and 4 move half a
// step, so some lane of nearly every warp enters a new cell there, and they enter it without the
// test (F::at_enter: the same cell, fractions and values).
template <typename T, class F>
__device__ __forceinline__ void rk4_increment_cell(const F &f, typename F::Cell &cell, T c, T ip,
                                                   const T y[6], T h, T inc[6])
{
    rk4_stages<T>(
        [&](int st, T x0, T x1, T x2, T &bx, T &by, T &bz) {
            if (st & 1)
                f.at_enter(cell, x0, x1, x2, bx, by, bz);
            else
                f.at_cell(cell, x0, x1, x2, bx, by, bz);
        },
        c, ip, y, h, inc);
}

template <typename T, class F>
__device__ __forceinline__ void rk4_step(const F &f, T c, T ip, T y[6], T h)
{
    T inc[6];
    rk4_increment<T, F>(f, c, ip, y, h, inc);
#pragma unroll
    for (int i = 0; i < 6; ++i) y[i] += inc[i];
}

// hi + lo += d, renormalised so that |lo| <= ulp(hi)/2 (Knuth's TwoSum; the rounded adds are never
// contracted or reassociated).
__device__ __forceinline__ void two_sum_add(float &hi, float &lo, float d)
{
    const float t = __fadd_rn(d, lo);
    const float s = __fadd_rn(hi, t);
    const float bb = __fsub_rn(s, hi);
    const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(t, bb));
    hi = s;
    lo = err;
}

// ------------------------------------------------------------------------------------------------
// Float-float arithmetic: a value is the unevaluated sum hi + lo of two floats (about 48 bits).
// Products use the exact FMA residual (TwoProd), sums Knuth's TwoSum; results are renormalised so
// that hi is the float nearest to the pair.  Used for per-seed constants of the FP32 path, which
// are then rounded to float once: on this part FP32 instructions are far cheaper than FP64 ones.
// ------------------------------------------------------------------------------------------------

__device__ __forceinline__ ff ff_renorm(float s, float e)   // |e| small against |s| (or s = 0)
{
    const float h = __fadd_rn(s, e);
    return ff{h, __fsub_rn(e, __fsub_rn(h, s))};
}

__device__ __forceinline__ ff ff_add(ff x, ff y)
{
    const float s = __fadd_rn(x.hi, y.hi);
    const float v = __fsub_rn(s, x.hi);
    float e = __fadd_rn(__fsub_rn(x.hi, __fsub_rn(s, v)), __fsub_rn(y.hi, v));
    e = __fadd_rn(e, __fadd_rn(x.lo, y.lo));
    return ff_renorm(s, e);
}

__device__ __forceinline__ ff ff_neg(ff x) { return ff{-x.hi, -x.lo}; }
__device__ __forceinline__ ff ff_sub(ff x, ff y) { return ff_add(x, ff_neg(y)); }

__device__ __forceinline__ ff ff_mul(ff x, ff y)
{
    const float p = __fmul_rn(x.hi, y.hi);
    float e = __fmaf_rn(x.hi, y.hi, -p);
    e = __fmaf_rn(x.hi, y.lo, e);
    e = __fmaf_rn(x.lo, y.hi, e);
    return ff_renorm(p, e);
}

__device__ __forceinline__ ff ff_mulf(ff x, float b)
{
    const float p = __fmul_rn(x.hi, b);
    float e = __fmaf_rn(x.hi, b, -p);
    e = __fmaf_rn(x.lo, b, e);
    return ff_renorm(p, e);
}

// 1 / x: one Newton step r + r (1 - x r) from the float reciprocal, the residual in float-float.
__device__ __forceinline__ ff ff_recip(ff x)
{
    const float r = __frcp_rn(x.hi);
    const ff e = ff_sub(ff{1.f, 0.f}, ff_mulf(x, r));
    return ff_add(ff{r, 0.f}, ff_mulf(e, r));
}

// sqrt(x), x > 0: one Newton step s + (x - s^2) / (2 s) from the float square root.
__device__ __forceinline__ ff ff_sqrt(ff x)
{
    const float s = __fsqrt_rn(x.hi);
    const float p = __fmul_rn(s, s);
    const ff d = ff_sub(x, ff{p, __fmaf_rn(s, s, -p)});
    return ff_renorm(s, __fdiv_rn(d.hi, __fmul_rn(2.f, s)));
}

// Exact float-float value of a double (host-side or constant operands).
__host__ __device__ constexpr ff ff_of(double v)
{
    return ff{(float)v, (float)(v - (double)(float)v)};
}

// hi + lo + d as a new pair by Fast2Sum (3 additions fewer than TwoSum): exact whenever |hi| is at
// least |d + lo| in exponent; when a component passes through zero it is off by at most about
// ulp(d), i.e. ~2e-9 m for a 16 mm step or ~5e-7 MeV/c for a 5 MeV/c one, a few times per turn.
__device__ __forceinline__ void fast_two_sum_add(float &hi, float &lo, float d)
{
    const float t = __fadd_rn(d, lo);
    const float s = __fadd_rn(hi, t);
    lo = __fsub_rn(t, __fsub_rn(s, hi));
    hi = s;
}

// c = KAPPA q / P0 and 1 / P0 of a seed from its recorded momentum (state 0), in the working
// precision; the DCA and classification kernels use the same helper, hence the same values.
template <typename T>
__device__ __forceinline__ void seed_kinematics(T px, T py, T pz, int q, T &c, T &ip)
{
    const T P0 = sqrt(px * px + py * py + pz * pz);
    ip = T(1) / P0;
    c = T(kKappa) * T(q) * ip;
}

// ------------------------------------------------------------------------------------------------
// Geometry
// ------------------------------------------------------------------------------------------------

// Squared distance of (x, y, z) to the line through a with unit direction u.
template <typename T>
__device__ __forceinline__ T line_dist2(T x, T y, T z, T ax, T ay, T az, T ux, T uy, T uz)
{
    const T dx = x - ax, dy = y - ay, dz = z - az;
    const T t = dx * ux + dy * uy + dz * uz;
    const T ex = dx - t * ux, ey = dy - t * uy, ez = dz - t * uz;
    return ex * ex + ey * ey + ez * ez;
}

// Orthonormal frame of a wire: unit vectors v, w perpendicular to its direction u, and the
// projections of its point a on them.  The squared distance of x to the wire line is then
// (x.v - a.v)^2 + (x.w - a.w)^2: two dot products.  Computed in the working precision from (a, u)
// by the same code in every kernel that searches for the closest recorded state, so they all get
// identical frames (the search bounds carry margins for its rounding).
template <typename T>
struct WireFrame {
    T vx, vy, vz, wx, wy, wz, av, aw;
};

template <typename T>
__device__ __forceinline__ WireFrame<T> wire_frame(T ax, T ay, T az, T ux, T uy, T uz)
{
    // helper axis least aligned with u
    T ex = T(0), ey = T(0), ez = T(0);
    const T fx = fabs(ux), fy = fabs(uy), fz = fabs(uz);
    if (fx <= fy && fx <= fz)
        ex = T(1);
    else if (fy <= fz)
        ey = T(1);
    else
        ez = T(1);
    const T eu = ex * ux + ey * uy + ez * uz;
    T vx = ex - eu * ux, vy = ey - eu * uy, vz = ez - eu * uz;
    const T vn = T(1) / sqrt(vx * vx + vy * vy + vz * vz);
    vx *= vn;
    vy *= vn;
    vz *= vn;
    WireFrame<T> f;
    f.vx = vx;
    f.vy = vy;
    f.vz = vz;
    f.wx = uy * vz - uz * vy;
    f.wy = uz * vx - ux * vz;
    f.wz = ux * vy - uy * vx;
    f.av = ax * f.vx + ay * f.vy + az * f.vz;
    f.aw = ax * f.wx + ay * f.wy + az * f.wz;
    return f;
}

// Distance form of the closest-state search (dca and classify use the same one, so that they pick the
// same state): 1 = the wire frame (8 FP ops), 0 = the difference form line_dist2 (12 FP ops).
#ifndef COMET_SEARCH_FRAME
#define COMET_SEARCH_FRAME 1
#endif

// Squared distance of (x, y, z) to the wire line in the wire's frame.
template <typename T>
__device__ __forceinline__ T frame_dist2(T x, T y, T z, T vx, T vy, T vz, T av, T wx, T wy, T wz,
                                         T aw)
{
    const T p = fma(x, vx, fma(y, vy, fma(z, vz, -av)));
    const T q = fma(x, wx, fma(y, wy, fma(z, wz, -aw)));
    return fma(p, p, q * q);
}

template <typename T>
__device__ __forceinline__ T rsqrt_t(T v);
template <>
__device__ __forceinline__ float rsqrt_t<float>(float v) { return rsqrtf(v); }
template <>
__device__ __forceinline__ double rsqrt_t<double>(double v) { return 1.0 / sqrt(v); }

// Lexicographic (distance, index) minimum: the lowest index wins exact ties.
template <typename T>
__device__ __forceinline__ void lex_min(T &bd, int &bk, T d, int k)
{
    if (d < bd || (d == bd && k < bk)) {
        bd = d;
        bk = k;
    }
}

// Virtual-plane refinement of Algorithm 2 from state y: the plane contains the wire axis and has
// normal n = t - (t.u) u (t the unit direction); d is the state's signed distance to it.  While
// |d| >= tol, step along the track by -d/|n| with one RK4 step (moving ds along the track moves the
// state |n| ds towards the plane).  The search is local: the state moves at most h_rec (one
// recording interval) along the track from where it started, which brackets the distance minimum
// of the starting state's valley; a step is shortened to stay inside.  Returns 1 if |d| < tol was
// reached within max_iter steps, 0 if not, if the track runs parallel to the wire, or if the state
// is held at the edge of the interval.  D = distance of the final state to the wire line.
// s0 != 0 takes a first step of that length (|s0| <= h_rec; it counts as one of the max_iter steps)
// before the first evaluation: a better start than the recorded state, the same fixed point.
template <typename T, class F>
__device__ __forceinline__ int refine_dca(const F &f, T c, T ip, T y[6], T ax, T ay, T az, T ux,
                                          T uy, T uz, T tol, int max_iter, T h_rec, T &D,
                                          T s0 = T(0))
{
    int conv = 0;
    T sigma = T(0);
    int it0 = 0;
    if (s0 != T(0)) {
        rk4_step<T, F>(f, c, ip, y, s0);
        sigma = s0;
        it0 = 1;
    }
    for (int it = it0;; ++it) {
        // t = p / P0: |p| stays P0 in a magnetic field, and the plane and its zero do not depend on
        // the norm of t (n is normalised below), only the Newton step length, by rounding
        const T tx = y[3] * ip, ty = y[4] * ip, tz = y[5] * ip;
        const T tu = tx * ux + ty * uy + tz * uz;
        const T nx = tx - tu * ux, ny = ty - tu * uy, nz = tz - tu * uz;
        const T nn2 = nx * nx + ny * ny + nz * nz;
        if (nn2 < T(1e-18)) break;
        const T rn = rsqrt_t<T>(nn2);
        const T dist = ((y[0] - ax) * nx + (y[1] - ay) * ny + (y[2] - az) * nz) * rn;
        if (fabs(dist) < tol) {
            conv = 1;
            break;
        }
        if (it >= max_iter) break;
        T target = sigma - dist * rn;
        target = target > h_rec ? h_rec : target;
        target = target < -h_rec ? -h_rec : target;
        const T ds = target - sigma;
        if (ds == T(0)) break;
        rk4_step<T, F>(f, c, ip, y, ds);
        sigma = target;
    }
    D = sqrt(line_dist2<T>(y[0], y[1], y[2], ax, ay, az, ux, uy, uz));
    return conv;
}

// ------------------------------------------------------------------------------------------------
// Bounding spheres of track segments (closest-state search)
// ------------------------------------------------------------------------------------------------

// The recorded states of a seed are cut into at most kN0Max super-segments of G0 states, each cut
// into at most kN1Max level-1 segments of G1 states.  For every group of 32 consecutive seeds (one
// warp) the search keeps one bounding sphere per segment: kBoundsPerGroup float4 (x, y, z, radius),
// super-segment j at [j], level-1 segment (j, m) at [kN0Max + j * kN1Max + m]; radius < 0 marks a
// segment no seed of the group has.
constexpr int kN0Max = 8;
constexpr int kN1Max = 24;
constexpr int kBoundsPerGroup = kN0Max + kN0Max * kN1Max;

// Centre index of a lane's segment [st, st + g) inside [.., end) (end = its last state + 1).
__device__ __forceinline__ int segment_centre(int st, int g, int end) { return min(st + g / 2, min(st + g, end) - 1); }

// The warp's bounding sphere of one segment: lanes with `has` hold their seed's segment centre
// (x, y, z); the sphere is centred on the midpoint of the first and the last such lane's centres
// (opposite corners of the lattice block, so about the middle of the group's tracks), its radius
// is the largest distance to any lane's centre plus `reach` (a state within g/2 recording intervals
// of a centre is at most (g/2) h_rec from it along the track).  Any centre gives a valid sphere;
// the radius is measured from the centre as rounded, and rounded up so that it never shrinks; in
// double the rounding of the centre to float is added.  Returns radius < 0 when no lane has the
// segment.
template <typename T>
__device__ __forceinline__ float4 warp_sphere(bool has, T x, T y, T z, T reach)
{
    const uint32_t hm = __ballot_sync(0xffffffffu, has);
    if (hm == 0u) return make_float4(0.f, 0.f, 0.f, -1.f);
    const int l0 = __ffs(hm) - 1, l1 = 31 - __clz(hm);
    const T cx = T(0.5) * (__shfl_sync(0xffffffffu, x, l0) + __shfl_sync(0xffffffffu, x, l1));
    const T cy = T(0.5) * (__shfl_sync(0xffffffffu, y, l0) + __shfl_sync(0xffffffffu, y, l1));
    const T cz = T(0.5) * (__shfl_sync(0xffffffffu, z, l0) + __shfl_sync(0xffffffffu, z, l1));
    // d^2 >= 0 as a float (rounded up from double): its bit pattern orders like its value, so one
    // integer warp reduction finds the max; then one root by the hardware reciprocal square root
    // (a few ulp, inside the 1e-6 relative margin below).  The radius is a float either way, so the
    // double path needs no double root or reductions (this part's FP64 rate is small).
    float d2;
    if constexpr (sizeof(T) == 4)
        d2 = has ? (x - cx) * (x - cx) + (y - cy) * (y - cy) + (z - cz) * (z - cz) : 0.f;
    else
        d2 = has ? __double2float_ru((x - cx) * (x - cx) + (y - cy) * (y - cy) + (z - cz) * (z - cz)) : 0.f;
    const float m2 = __uint_as_float(__reduce_max_sync(0xffffffffu, __float_as_uint(d2)));
    const T d = (T)(m2 * rsqrtf(fmaxf(m2, 1e-30f)));
    const T extra = sizeof(T) == 8 ? T(2e-7) : T(0);
    return make_float4((float)cx, (float)cy, (float)cz, (float)((d + reach + extra) * T(1.000001)));
}

// ------------------------------------------------------------------------------------------------
// Shared-memory staging with the bulk-copy engine (cp.async.bulk + mbarrier)
// ------------------------------------------------------------------------------------------------

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
            "r"(smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// Orders this thread's earlier generic-proxy shared-memory accesses before later bulk copies.
__device__ __forceinline__ void fence_proxy_async_smem()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ uint64_t global_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Waits for phase `parity` of the barrier to complete, for at most ~timeout_ns.  Returns false on
// timeout (the caller then records an error and falls back to plain loads).
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, uint64_t timeout_ns)
{
    const uint32_t a = smem_u32(bar);
    const uint64_t t0 = global_ns();
    for (uint32_t it = 0; it < (1u << 26); ++it) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
            " selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
        if ((it & 63) == 63 && global_ns() - t0 > timeout_ns) return false;
    }
    return false;
}

// Plan for copying n elements of size es from global src into a 16-byte-aligned shared buffer so
// that element i lands at dst[off + i]: the 16-byte-aligned middle goes through one bulk copy, the
// ragged head and tail through plain loads.  Every thread computes the same plan from the address.
struct StagePlan {
    int off;      // element offset of element 0 inside the shared buffer
    int head;     // elements before the first 16-byte boundary of src
    int body;     // elements in the bulk-copied middle
};

__device__ __forceinline__ StagePlan stage_plan(const void *src, int n, int es)
{
    StagePlan p;
    const int mis = (int)((uintptr_t)src & 15);
    p.off = mis / es;
    int head = mis == 0 ? 0 : (16 - mis) / es;
    head = head > n ? n : head;
    p.head = head;
    p.body = (((n - head) * es) / 16) * 16 / es;
    return p;
}

} // namespace comet
