// Residual Jacobians for Gauss-Newton refinement of the best seeds (FP64, uniform axial field).
//
// The seed is parameterised by theta = (z0, phi, pz, pT) with the vertex (vx, vy) fixed, as in the
// lattice.  With P = px + i py and X = x + i y, one RK4 step of length h in B = (0, 0, Bz) is the
// linear map P' = m P, X' = X + n P, z' = z + dz, whose coefficients depend on P0 = |p| and h only
// (device.cuh); the k-th recorded state is therefore P_k = M^k P_0, X_k = X_0 + N (M^k - 1)/(M - 1)
// P_0 with (M, N) the map of one recording interval.  Carrying every quantity as a value plus its
// four partial derivatives in theta (forward mode) gives the derivatives of the recorded states in
// closed form.
//
// The DCA of a wire is the distance at the point of closest approach (PCA) found as in the scan: the
// closest recorded state (searched in FP32, settled in FP64 among its neighbours), then the local
// virtual-plane Newton refinement of Algorithm 2, each refinement step being one RK4 step of the
// axial map.  At the PCA the distance
// is stationary along the track, so dD/dtheta = nhat . dx/dtheta at the fixed arc length of the PCA
// (envelope theorem): the refinement steps are replayed in forward mode with their lengths held
// fixed.  nhat is the unit vector from the wire to the PCA.
//
// Smoothed residual (Eq. 1 with a differentiable cap): e = min_j |D - r_j| over the wire's unmasked
// hits, w = sigmoid((lambda - e) / tau), term = w e^2 + (1 - w) lambda^2.  Gauss-Newton treats w as
// fixed within an iteration: residual rho = D - r_j* with weight w.
#include <math.h>

#include "device.cuh"
#include "internal.h"

namespace comet {

namespace {

// value + 4 partial derivatives
struct D4 {
    double v, d[4];
};

__device__ __forceinline__ D4 dc(double v) { return D4{v, {0.0, 0.0, 0.0, 0.0}}; }
__device__ __forceinline__ D4 operator+(const D4 &a, const D4 &b)
{
    return D4{a.v + b.v, {a.d[0] + b.d[0], a.d[1] + b.d[1], a.d[2] + b.d[2], a.d[3] + b.d[3]}};
}
__device__ __forceinline__ D4 operator-(const D4 &a, const D4 &b)
{
    return D4{a.v - b.v, {a.d[0] - b.d[0], a.d[1] - b.d[1], a.d[2] - b.d[2], a.d[3] - b.d[3]}};
}
__device__ __forceinline__ D4 operator-(const D4 &a) { return D4{-a.v, {-a.d[0], -a.d[1], -a.d[2], -a.d[3]}}; }
__device__ __forceinline__ D4 operator*(const D4 &a, const D4 &b)
{
    D4 r;
    r.v = a.v * b.v;
#pragma unroll
    for (int j = 0; j < 4; ++j) r.d[j] = a.d[j] * b.v + a.v * b.d[j];
    return r;
}
__device__ __forceinline__ D4 operator*(double s, const D4 &a)
{
    return D4{s * a.v, {s * a.d[0], s * a.d[1], s * a.d[2], s * a.d[3]}};
}
__device__ __forceinline__ D4 operator/(const D4 &a, const D4 &b)
{
    D4 r;
    const double ib = 1.0 / b.v;
    r.v = a.v * ib;
#pragma unroll
    for (int j = 0; j < 4; ++j) r.d[j] = (a.d[j] - r.v * b.d[j]) * ib;
    return r;
}
__device__ __forceinline__ D4 dsqrt(const D4 &a)
{
    D4 r;
    r.v = sqrt(a.v);
    const double k = r.v > 0.0 ? 0.5 / r.v : 0.0;
#pragma unroll
    for (int j = 0; j < 4; ++j) r.d[j] = a.d[j] * k;
    return r;
}

// complex number of D4 parts
struct C4 {
    D4 re, im;
};
__device__ __forceinline__ C4 operator+(const C4 &a, const C4 &b) { return C4{a.re + b.re, a.im + b.im}; }
__device__ __forceinline__ C4 operator*(const C4 &a, const C4 &b)
{
    return C4{a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
__device__ __forceinline__ C4 cdiv(const C4 &a, const C4 &b)
{
    const D4 den = b.re * b.re + b.im * b.im;
    return C4{(a.re * b.re + a.im * b.im) / den, (a.im * b.re - a.re * b.im) / den};
}

// One RK4 step of length h in the axial field: P' = m P, X' = X + n P, z' = z + dz, with m = 1 + A.
struct StepMap {
    C4 A, n;   // A = m - 1 = am1 - i b, n = c - i d
    D4 dz;
};

__device__ __forceinline__ StepMap step_map(const D4 &P0, const D4 &pz, double h, double kqb)
{
    const D4 ip = dc(1.0) / P0;
    const D4 t = (h * kqb) * ip;
    const D4 t2 = t * t;
    const D4 hp = h * ip;
    const D4 g = dc(1.0) - (1.0 / 6.0) * t2;
    StepMap s;
    s.A.re = t2 * (dc(-0.5) + (1.0 / 24.0) * t2);
    s.A.im = -(t * g);
    s.n.re = hp * g;
    s.n.im = -(hp * t * (dc(0.5) - (1.0 / 24.0) * t2));
    s.dz = hp * pz;
    return s;
}

// (1 + A)^k - 1 by binary powering on A ((1 + a)(1 + b) - 1 = a + b + a b: nothing cancels)
__device__ __forceinline__ C4 pow_minus_one(const C4 &A, int k)
{
    C4 R{dc(0.0), dc(0.0)}, Bp = A;
    bool first = true;
    for (int e = k; e > 0; e >>= 1) {
        if (e & 1) {
            if (first) {
                R = Bp;
                first = false;
            } else {
                R = R + Bp + R * Bp;
            }
        }
        if (e > 1) Bp = Bp + Bp + Bp * Bp;
    }
    return R;
}

// k steps of a map (same coefficients): A_k = (1 + A)^k - 1, n_k = n (A_k / A), dz_k = k dz
__device__ __forceinline__ StepMap power_map(const StepMap &s, int k)
{
    StepMap r;
    r.A = pow_minus_one(s.A, k);
    const bool turns = s.A.re.v != 0.0 || s.A.im.v != 0.0;
    const C4 S = turns ? cdiv(r.A, s.A) : C4{dc((double)k), dc(0.0)};
    r.n = s.n * S;
    r.dz = (double)k * s.dz;
    return r;
}

struct State4 {
    C4 X, P;
    D4 z;
};

__device__ __forceinline__ State4 apply(const StepMap &s, const State4 &y)
{
    State4 o;
    o.X = y.X + s.n * y.P;
    o.P = y.P + s.A * y.P;
    o.z = y.z + s.dz;
    return o;
}

// value-only version of a step: (x, y, z, px, py) += the map
struct Step1 {
    double am1, b, c, d, dz;
};
__device__ __forceinline__ Step1 step1(double P0, double pz, double h, double kqb)
{
    const double t = h * kqb / P0, t2 = t * t, hp = h / P0, g = 1.0 - t2 / 6.0;
    return Step1{t2 * (-0.5 + t2 / 24.0), t * g, hp * g, hp * t * (0.5 - t2 / 24.0), hp * pz};
}
__device__ __forceinline__ void apply1(const Step1 &s, double y[5])
{
    const double px = y[3], py = y[4];
    y[0] += s.c * px + s.d * py;
    y[1] += s.c * py - s.d * px;
    y[2] += s.dz;
    y[3] += s.am1 * px + s.b * py;
    y[4] += s.am1 * py - s.b * px;
}

constexpr int kMaxSteps = 64;   // refinement steps replayed in forward mode (max_iter is capped)

__global__ void __launch_bounds__(32) jacobian_kernel(JacArgs a)
{
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (tid >= a.S * a.W) return;
    const int64_t s = tid / a.W;
    const int i = (int)(tid % a.W);
    double *out = a.work + tid * 11;   // flag, term, dterm, w, rho, J[0..3], nhat_x, nhat_y
    const int hb = a.offs[i], he = a.offs[i + 1];
    bool any = false;
    for (int j = hb; j < he; ++j) any = any || !a.mask[j];

    // seed and its derivatives: theta = (z0, phi, pz, pT)
    const double *th = a.theta + s * 4;
    const double cphi = cos(th[1]), sphi = sin(th[1]);
    State4 y0;
    y0.X = C4{dc(a.vx), dc(a.vy)};
    y0.P.re = D4{th[3] * cphi, {0.0, -th[3] * sphi, 0.0, cphi}};
    y0.P.im = D4{th[3] * sphi, {0.0, th[3] * cphi, 0.0, sphi}};
    y0.z = D4{th[0], {1.0, 0.0, 0.0, 0.0}};
    const D4 pz = D4{th[2], {0.0, 0.0, 1.0, 0.0}};
    const D4 pt = D4{th[3], {0.0, 0.0, 0.0, 1.0}};
    const D4 P0 = dsqrt(pt * pt + pz * pz);
    const double kqb = kKappa * a.charge * a.bz;
    const StepMap one = step_map(P0, pz, a.h, kqb);
    const StepMap itv = power_map(one, a.stride);

    // wire
    const double *w = (const double *)a.wires;
    const double ax = w[0 * a.ldw + i], ay = w[1 * a.ldw + i], az = w[2 * a.ldw + i];
    const double ux = w[3 * a.ldw + i], uy = w[4 * a.ldw + i], uz = w[5 * a.ldw + i];

    // closest recorded state, recording as the scan does: state 0, then each interval, stopping
    // after the first state outside the target region.  The walk runs in FP32 (FP64 instructions
    // are scarce on this part); the argmin is then settled in FP64 among the FP32 choice and its
    // two neighbours.
    const double pzv = pz.v;
    const float am1f = (float)itv.A.re.v, bbf = (float)-itv.A.im.v, ccf = (float)itv.n.re.v,
                ddf = (float)-itv.n.im.v, dzf = (float)itv.dz.v;
    float f[5] = {(float)y0.X.re.v, (float)y0.X.im.v, (float)y0.z.v, (float)y0.P.re.v, (float)y0.P.im.v};
    const float axf = (float)ax, ayf = (float)ay, azf = (float)az, uxf = (float)ux, uyf = (float)uy,
                uzf = (float)uz;
    const float zminf = (float)a.zmin, zmaxf = (float)a.zmax, rmax2f = (float)a.rmax2;
    float bestf = INFINITY;
    int kbest = 0, nvalid = a.n_rec;
    for (int k = 0; k < a.n_rec; ++k) {
        if (k > 0) {
            const float px = f[3], py = f[4];
            f[0] += ccf * px + ddf * py;
            f[1] += ccf * py - ddf * px;
            f[2] += dzf;
            f[3] += am1f * px + bbf * py;
            f[4] += am1f * py - bbf * px;
        }
        const float d2 = line_dist2<float>(f[0], f[1], f[2], axf, ayf, azf, uxf, uyf, uzf);
        if (d2 < bestf) {
            bestf = d2;
            kbest = k;
        }
        if (f[2] < zminf || f[2] > zmaxf || f[0] * f[0] + f[1] * f[1] > rmax2f) {
            nvalid = k + 1;
            break;
        }
    }
    // FP64 (forward mode): states kbest - 1 .. kbest + 1, the lowest distance, ties to the lower index
    const int k0 = kbest > 0 ? kbest - 1 : 0;
    const State4 base = k0 > 0 ? apply(power_map(itv, k0), y0) : y0;
    {
        double best = INFINITY;
        int kb = kbest;
        State4 cur = base;
        for (int k = k0; k <= kbest + 1 && k < nvalid; ++k) {
            if (k > k0) cur = apply(itv, cur);
            const double d2 = line_dist2<double>(cur.X.re.v, cur.X.im.v, cur.z.v, ax, ay, az, ux, uy, uz);
            if (d2 < best) {
                best = d2;
                kb = k;
            }
        }
        kbest = kb;
    }
    State4 yk = base;
    for (int k = k0; k < kbest; ++k) yk = apply(itv, yk);

    // local virtual-plane refinement (values), remembering the step lengths
    double y[6] = {yk.X.re.v, yk.X.im.v, yk.z.v, yk.P.re.v, yk.P.im.v, pzv};
    double ds_list[kMaxSteps];
    int n_ds = 0, conv = 0;
    double sigma = 0.0;
    const int max_iter = a.max_iter < kMaxSteps ? a.max_iter : kMaxSteps;
    for (int it = 0;; ++it) {
        const double rp = 1.0 / sqrt(y[3] * y[3] + y[4] * y[4] + y[5] * y[5]);
        const double tx = y[3] * rp, ty = y[4] * rp, tz = y[5] * rp;
        const double tu = tx * ux + ty * uy + tz * uz;
        const double nx = tx - tu * ux, ny = ty - tu * uy, nz = tz - tu * uz;
        const double nn2 = nx * nx + ny * ny + nz * nz;
        if (nn2 < 1e-18) break;
        const double rn = 1.0 / sqrt(nn2);
        const double dist = ((y[0] - ax) * nx + (y[1] - ay) * ny + (y[2] - az) * nz) * rn;
        if (fabs(dist) < a.tol) {
            conv = 1;
            break;
        }
        if (it >= max_iter) break;
        double target = sigma - dist * rn;
        target = target > a.h_rec ? a.h_rec : target;
        target = target < -a.h_rec ? -a.h_rec : target;
        const double ds = target - sigma;
        if (ds == 0.0) break;
        const Step1 st = step1(P0.v, pzv, ds, kqb);
        double y5[5] = {y[0], y[1], y[2], y[3], y[4]};
        apply1(st, y5);
        for (int c = 0; c < 5; ++c) y[c] = y5[c];
        ds_list[n_ds++] = ds;
        sigma = target;
    }
    // replay the steps in forward mode at their fixed lengths
    for (int q = 0; q < n_ds; ++q) yk = apply(step_map(P0, pz, ds_list[q], kqb), yk);

    // D and dD/dtheta = nhat . dx/dtheta
    const double rx = yk.X.re.v - ax, ry = yk.X.im.v - ay, rz = yk.z.v - az;
    const double al = rx * ux + ry * uy + rz * uz;
    const double ex = rx - al * ux, ey = ry - al * uy, ez = rz - al * uz;
    const double D = sqrt(ex * ex + ey * ey + ez * ez);
    const double inv = D > 0.0 ? 1.0 / D : 0.0;
    double J[4];
#pragma unroll
    for (int j = 0; j < 4; ++j)
        J[j] = (ex * yk.X.re.d[j] + ey * yk.X.im.d[j] + ez * yk.z.d[j]) * inv;

    // smoothed residual of the wire
    double term = 0.0, dterm = 0.0, wgt = 0.0, rho = 0.0;
    if (any) {
        double e = INFINITY, r_best = 0.0;
        for (int j = hb; j < he; ++j) {
            if (a.mask[j]) continue;
            const double ej = fabs(D - a.drift[j]);
            if (ej < e) {
                e = ej;
                r_best = a.drift[j];
            }
        }
        const double lam = a.lambda;
        wgt = 1.0 / (1.0 + exp(-(lam - e) / a.tau));
        term = wgt * e * e + (1.0 - wgt) * lam * lam;
        const double dw = -wgt * (1.0 - wgt) / a.tau;
        const double sgn = D >= r_best ? 1.0 : -1.0;
        dterm = sgn * (2.0 * wgt * e + dw * (e * e - lam * lam));
        rho = D - r_best;
    }
    out[0] = any ? 1.0 : 0.0;
    out[1] = term;
    out[2] = dterm;
    out[3] = wgt;
    out[4] = rho;
    if (a.dca_out) a.dca_out[tid] = D;
    if (a.jac_out) {
#pragma unroll
        for (int j = 0; j < 4; ++j) a.jac_out[tid * 4 + j] = J[j];
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) out[5 + j] = J[j];
    out[9] = ex * inv;    // dD/dx0 and dD/dy0: the recorded X_k depend on (x0, y0) additively
    out[10] = ey * inv;
    if (!conv && any && a.n_unconv) atomicAdd(a.n_unconv, 1);
}

// per seed, ascending wire order: smoothed RSS, its gradient, J^T W J and J^T W rho
__global__ void jacobian_reduce_kernel(JacArgs a)
{
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= a.S) return;
    double srss = 0.0, g[4] = {0, 0, 0, 0}, jtj[16], jtr[4] = {0, 0, 0, 0}, gxy[2] = {0, 0};
    for (int q = 0; q < 16; ++q) jtj[q] = 0.0;
    for (int i = 0; i < a.W; ++i) {
        const int64_t t = s * a.W + i;
        const double *o = a.work + t * 11;
        if (o[0] == 0.0) continue;
        const double *J = o + 5;
        srss += o[1];
        gxy[0] += o[2] * o[9];
        gxy[1] += o[2] * o[10];
        for (int j = 0; j < 4; ++j) {
            g[j] += o[2] * J[j];
            jtr[j] += o[3] * o[4] * J[j];
            for (int k = 0; k < 4; ++k) jtj[j * 4 + k] += o[3] * J[j] * J[k];
        }
    }
    a.srss_out[s] = srss;
    for (int j = 0; j < 4; ++j) {
        a.grad_out[s * 4 + j] = g[j];
        a.jtr_out[s * 4 + j] = jtr[j];
    }
    for (int q = 0; q < 16; ++q) a.jtj_out[s * 16 + q] = jtj[q];
    if (a.grad6_out) {
        // (x0, y0, z0, px, py, pz): phi = atan2(py, px) and pT = hypot(px, py), by the chain rule
        const double phi = a.theta[s * 4 + 1], pt = a.theta[s * 4 + 3];
        const double cp = cos(phi), sp = sin(phi);
        double *o = a.grad6_out + s * 6;
        o[0] = gxy[0];
        o[1] = gxy[1];
        o[2] = g[0];
        o[3] = -g[1] * sp / pt + g[3] * cp;
        o[4] = g[1] * cp / pt + g[3] * sp;
        o[5] = g[2];
    }
}

// Solves (J^T W J + mu diag(J^T W J)) x = -J^T W rho for one seed by Cholesky; returns false (x
// untouched) when the damped matrix is not positive definite.
__device__ bool damped_normal_solve(const double *jtj, const double *jtr, double mu, double x[4])
{
    double A[4][4], L[4][4] = {}, r[4];
    for (int j = 0; j < 4; ++j) {
        for (int k = 0; k < 4; ++k) A[j][k] = jtj[j * 4 + k];
        A[j][j] *= 1.0 + mu;
        r[j] = -jtr[j];
    }
    for (int j = 0; j < 4; ++j) {
        double d = A[j][j];
        for (int k = 0; k < j; ++k) d -= L[j][k] * L[j][k];
        if (!(d > 0.0)) return false;
        L[j][j] = sqrt(d);
        for (int i = j + 1; i < 4; ++i) {
            double v = A[i][j];
            for (int k = 0; k < j; ++k) v -= L[i][k] * L[j][k];
            L[i][j] = v / L[j][j];
        }
    }
    double z[4];
    for (int j = 0; j < 4; ++j) {
        double v = r[j];
        for (int k = 0; k < j; ++k) v -= L[j][k] * z[k];
        z[j] = v / L[j][j];
    }
    for (int j = 3; j >= 0; --j) {
        double v = z[j];
        for (int k = j + 1; k < 4; ++k) v -= L[k][j] * x[k];
        x[j] = v / L[j][j];
    }
    return true;
}

// theta += delta, (J^T W J + mu diag(J^T W J)) delta = -J^T W rho, by Cholesky; a seed whose
// matrix is not positive definite keeps its theta
__global__ void gn_step_kernel(double *theta, int64_t S, const double *jtj, const double *jtr, double mu)
{
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= S) return;
    double x[4];
    if (!damped_normal_solve(jtj + s * 16, jtr + s * 4, mu, x)) return;
    for (int j = 0; j < 4; ++j) theta[s * 4 + j] += x[j];
}

// Levenberg-Marquardt bookkeeping of one seed: judge the trial (accept it when its smoothed RSS is
// lower: it becomes the current seed with its normal equations, and the damping shrinks; else the
// damping grows), then form the next trial from the current seed.
__global__ void lm_step_kernel(LmArgs a)
{
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= a.S) return;
    double mu = a.mu[s];
    if (!a.first) {
        const double ft = a.srss_try[s];
        if (ft < a.srss[s]) {
            a.srss[s] = ft;
            for (int j = 0; j < 4; ++j) a.theta[s * 4 + j] = a.theta_try[s * 4 + j];
            for (int j = 0; j < 4; ++j) a.jtr[s * 4 + j] = a.jtr_try[s * 4 + j];
            for (int j = 0; j < 16; ++j) a.jtj[s * 16 + j] = a.jtj_try[s * 16 + j];
            mu = fmax(mu * a.down, a.mu_min);
        } else {
            mu = fmin(mu * a.up, a.mu_max);
        }
        a.mu[s] = mu;
    }
    double x[4] = {0.0, 0.0, 0.0, 0.0};
    damped_normal_solve(a.jtj + s * 16, a.jtr + s * 4, mu, x);
    for (int j = 0; j < 4; ++j) a.theta_try[s * 4 + j] = a.theta[s * 4 + j] + x[j];
}

} // namespace

cudaError_t launch_jacobian(const JacArgs &a, cudaStream_t st)
{
    const int64_t n = a.S * a.W;
    if (n > 0) {
        // small blocks: a few thousand threads of long FP64 chains, spread over as many SMs as possible
        jacobian_kernel<<<(unsigned)((n + 31) / 32), 32, 0, st>>>(a);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    jacobian_reduce_kernel<<<(unsigned)((a.S + 63) / 64), 64, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_gn_step(double *theta, int64_t S, const double *jtj, const double *jtr, double mu,
                           cudaStream_t st)
{
    gn_step_kernel<<<(unsigned)((S + 63) / 64), 64, 0, st>>>(theta, S, jtj, jtr, mu);
    return cudaGetLastError();
}

cudaError_t launch_lm_step(const LmArgs &a, cudaStream_t st)
{
    lm_step_kernel<<<(unsigned)((a.S + 63) / 64), 64, 0, st>>>(a);
    return cudaGetLastError();
}

} // namespace comet
