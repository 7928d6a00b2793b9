/*
 * FP64 CPU oracle of the brute-force seed scan (arXiv:1911.09340).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously-correct statement of what the
 * scan computes, used to check the CUDA library.  Only the tests, the smoke check and the bench's
 * CPU-baseline / reference leg may load it; the library never calls it and shares no code with it.
 *
 * What it computes, in the paper's order:
 *   - seed lattice: the Cartesian product of prior ranges of the seed components (Sec. 2.1, Sec. 3.1);
 *   - track recording (Algorithm 1): extrapolate each seed through the field and record its states,
 *     here with classic fixed-step RK4 (the paper uses adaptive RKN; the step is fixed here);
 *   - DCA finding (Algorithm 2, Sec. 2.2.2): for each wire, start from the recorded state closest to
 *     the wire line and step along the track by the distance to the virtual plane (which contains the
 *     wire axis) until that distance is under the tolerance; the DCA is the distance to the wire line;
 *   - RSS (Eq. 1): per wire the smallest |DCA - r| over its hits, capped at lambda, squared and summed
 *     in ascending wire order.  One CPU thread per seed, as Algorithm 3 does;
 *   - selection: seeds ordered by RSS (ties: lowest index) (Sec. 2.1);
 *   - classification (Sec. 2.1): for the selected seed, the closest hit of each wire is classified
 *     when its min(d^L, d^R) = |DCA - r| is below lambda.
 *
 * Equations of motion (units m, MeV/c, T): with arc length s, P0 = |p| of the seed and
 * KAPPA = 299.792458 MeV/c per (T m),
 *     dx/ds = p / P0,      dp/ds = (KAPPA q / P0) p x B(x).
 *
 * Layouts (all row-major, doubles unless stated): seeds [S][6] = (x, y, z, px, py, pz);
 * points [S][n_rec][6]; wires [W][6] = (a_x, a_y, a_z, u_x, u_y, u_z) with |u| = 1; hit_offsets
 * [W+1] (CSR into drift[H] and mask[H]); mask[H] = 1 marks a hit classified by an earlier turn
 * partition, which is then ignored.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define KAPPA 299.792458

typedef struct {
    int kind;              /* 0 uniform, 1 trilinear table */
    double b[3];           /* uniform field */
    const float *table;    /* [3][nz][ny][nx] */
    int nx, ny, nz;
    double origin[3];      /* position of node (0, 0, 0) */
    double spacing;        /* node spacing, same on all axes */
} or_field;

typedef struct {
    double h;              /* RK4 step (m) */
    int n_steps;           /* RK4 steps per partition */
    int stride;            /* record every stride-th state (state 0 is always recorded) */
    double lambda;         /* cutoff of Eq. 1 (m) */
    double tol;            /* virtual-plane distance tolerance (m) */
    int max_iter;          /* maximum refinement steps */
    double zmin, zmax, rmax;  /* recording stops once a recorded state is outside this region */
} or_params;

/* ---------------------------------------------------------------------------------------------- */
/* Field                                                                                          */
/* ---------------------------------------------------------------------------------------------- */

static double tab_at(const or_field *f, int c, int iz, int iy, int ix)
{
    size_t idx = (((size_t)c * f->nz + iz) * f->ny + iy) * f->nx + ix;
    return (double)f->table[idx];
}

/* Trilinear interpolation of the table; a coordinate outside the grid is clamped to its edge. */
static void field_at(const or_field *f, const double x[3], double B[3])
{
    if (f->kind == 0) {
        B[0] = f->b[0];
        B[1] = f->b[1];
        B[2] = f->b[2];
        return;
    }
    int n[3] = {f->nx, f->ny, f->nz};
    int i0[3];
    double t[3];
    for (int a = 0; a < 3; ++a) {
        double g = (x[a] - f->origin[a]) / f->spacing;
        if (g < 0.0) g = 0.0;
        if (g > (double)(n[a] - 1)) g = (double)(n[a] - 1);
        int i = (int)floor(g);
        if (i > n[a] - 2) i = n[a] - 2;
        i0[a] = i;
        t[a] = g - (double)i;
    }
    for (int c = 0; c < 3; ++c) {
        double v = 0.0;
        for (int dz = 0; dz < 2; ++dz)
            for (int dy = 0; dy < 2; ++dy)
                for (int dx = 0; dx < 2; ++dx) {
                    double w = (dx ? t[0] : 1.0 - t[0]) * (dy ? t[1] : 1.0 - t[1]) *
                               (dz ? t[2] : 1.0 - t[2]);
                    v += w * tab_at(f, c, i0[2] + dz, i0[1] + dy, i0[0] + dx);
                }
        B[c] = v;
    }
}

/* ---------------------------------------------------------------------------------------------- */
/* RK4 on y = (x, p)                                                                              */
/* ---------------------------------------------------------------------------------------------- */

static void deriv(const or_field *f, double q, double P0, const double y[6], double dy[6])
{
    double B[3];
    field_at(f, y, B);
    double c = KAPPA * q / P0;
    dy[0] = y[3] / P0;
    dy[1] = y[4] / P0;
    dy[2] = y[5] / P0;
    dy[3] = c * (y[4] * B[2] - y[5] * B[1]);
    dy[4] = c * (y[5] * B[0] - y[3] * B[2]);
    dy[5] = c * (y[3] * B[1] - y[4] * B[0]);
}

/* One classic fourth-order Runge-Kutta step of length h (h may be negative). */
static void rk4_step(const or_field *f, double q, double P0, double y[6], double h)
{
    double k1[6], k2[6], k3[6], k4[6], t[6];
    deriv(f, q, P0, y, k1);
    for (int i = 0; i < 6; ++i) t[i] = y[i] + 0.5 * h * k1[i];
    deriv(f, q, P0, t, k2);
    for (int i = 0; i < 6; ++i) t[i] = y[i] + 0.5 * h * k2[i];
    deriv(f, q, P0, t, k3);
    for (int i = 0; i < 6; ++i) t[i] = y[i] + h * k3[i];
    deriv(f, q, P0, t, k4);
    for (int i = 0; i < 6; ++i) y[i] += h / 6.0 * (k1[i] + 2.0 * k2[i] + 2.0 * k3[i] + k4[i]);
}

static int outside(const or_params *P, const double y[6])
{
    return y[2] < P->zmin || y[2] > P->zmax || y[0] * y[0] + y[1] * y[1] > P->rmax * P->rmax;
}

int oracle_n_rec(const or_params *P) { return P->n_steps / P->stride + 1; }

/* Track recording of one seed (Algorithm 1).  Writes up to n_rec states, returns how many. */
static int record_track(const or_field *f, const or_params *P, const double seed[6], int q,
                        double *pts /* [n_rec][6] */)
{
    double y[6];
    memcpy(y, seed, sizeof y);
    double P0 = sqrt(y[3] * y[3] + y[4] * y[4] + y[5] * y[5]);
    int n = 0;
    memcpy(pts, y, sizeof y);
    n = 1;
    if (outside(P, y)) return n;
    for (int step = 1; step <= P->n_steps; ++step) {
        rk4_step(f, (double)q, P0, y, P->h);
        if (step % P->stride == 0) {
            memcpy(pts + 6 * (size_t)n, y, sizeof y);
            ++n;
            if (outside(P, y)) break;
        }
    }
    return n;
}

/* ---------------------------------------------------------------------------------------------- */
/* DCA of one track to one wire (Algorithm 2 / Sec. 2.2.2)                                        */
/* ---------------------------------------------------------------------------------------------- */

/* Squared distance of point x to the line through a with unit direction u. */
static double line_dist2(const double x[3], const double w[6])
{
    double d[3] = {x[0] - w[0], x[1] - w[1], x[2] - w[2]};
    double t = d[0] * w[3] + d[1] * w[4] + d[2] * w[5];
    double e[3] = {d[0] - t * w[3], d[1] - t * w[4], d[2] - t * w[5]};
    return e[0] * e[0] + e[1] * e[1] + e[2] * e[2];
}

/* Returns the DCA; *converged is 0 when the refinement hit max_iter, met a track parallel to the
   wire, or was held at the edge of its search interval.  The refinement is local (Sec. 2.2: the
   closest recorded state "serves as a new seed to find the DCA within a few extrapolation steps"):
   the state moves at most one recording interval h_rec along the track from the closest recorded
   state, which brackets the distance minimum of that state's valley. */
static double dca_one(const or_field *f, const or_params *P, const double *pts, int n_valid,
                      int q, double P0, const double w[6], int *converged)
{
    /* closest recorded state (ties: lowest index) */
    int kbest = 0;
    double dbest = line_dist2(pts, w);
    for (int k = 1; k < n_valid; ++k) {
        double d2 = line_dist2(pts + 6 * (size_t)k, w);
        if (d2 < dbest) {
            dbest = d2;
            kbest = k;
        }
    }
    double y[6];
    memcpy(y, pts + 6 * (size_t)kbest, sizeof y);
    const double h_rec = P->h * P->stride;
    double sigma = 0.0;   /* arc length moved so far */
    *converged = 0;
    for (int it = 0;; ++it) {
        /* virtual plane: contains the wire axis, normal along the part of the track direction
           that is perpendicular to the wire */
        double pn = sqrt(y[3] * y[3] + y[4] * y[4] + y[5] * y[5]);
        double t[3] = {y[3] / pn, y[4] / pn, y[5] / pn};
        double tu = t[0] * w[3] + t[1] * w[4] + t[2] * w[5];
        double n[3] = {t[0] - tu * w[3], t[1] - tu * w[4], t[2] - tu * w[5]};
        double nn = sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
        if (nn < 1e-9) break;                     /* track parallel to the wire: no plane */
        double dist = ((y[0] - w[0]) * n[0] + (y[1] - w[1]) * n[1] + (y[2] - w[2]) * n[2]) / nn;
        if (fabs(dist) < P->tol) {
            *converged = 1;
            break;
        }
        if (it == P->max_iter) break;
        /* moving ds along the track moves the state nn*ds towards the plane */
        double target = sigma - dist / nn;
        if (target > h_rec) target = h_rec;
        if (target < -h_rec) target = -h_rec;
        double ds = target - sigma;
        if (ds == 0.0) break;                     /* held at the edge of the interval */
        rk4_step(f, (double)q, P0, y, ds);
        sigma = target;
    }
    return sqrt(line_dist2(y, w));
}

/* ---------------------------------------------------------------------------------------------- */
/* Public entry points (ctypes)                                                                   */
/* ---------------------------------------------------------------------------------------------- */

/* Seed lattice (Sec. 2.1: seeds combined from grids over the prior range of each component).
   Dimensions: z0, phi, pz, pt; node i of n sits at centre + half_width*(2i/(n-1) - 1).  The seed is
   (vx, vy, z0, pt cos phi, pt sin phi, pz).  Enumeration: the lattice is cut into blocks of
   b = (2, 4, 4, 1) nodes along (z0, phi, pz, pt) (z0: 1 when its count is odd; phi and pz: 2 when
   4 does not divide the count but 2 does, 1 when it is odd); blocks are numbered row-major (z0
   slowest) and the nodes inside a block row-major, so seed s = block * (b0 b1 b2 b3) +
   node-in-block. */
static int block_of(int n, int pref)
{
    if (pref >= 4 && n % 4 == 0) return 4;
    return n % 2 == 0 ? 2 : 1;
}

void oracle_block_shape(const int counts[4], int b[4])
{
    b[0] = block_of(counts[0], 2);
    b[1] = block_of(counts[1], 4);
    b[2] = block_of(counts[2], 4);
    b[3] = 1;
}

void oracle_lattice(double vx, double vy, const double centre[4], const double half_width[4],
                    const int counts[4], double *seeds /* [S][6] */)
{
    int b[4], nb[4];
    oracle_block_shape(counts, b);
    for (int d = 0; d < 4; ++d) nb[d] = counts[d] / b[d];
    int64_t vol = (int64_t)b[0] * b[1] * b[2] * b[3];
    int64_t S = (int64_t)counts[0] * counts[1] * counts[2] * counts[3];
    for (int64_t s = 0; s < S; ++s) {
        int64_t blk = s / vol, in = s % vol;
        int ii[4], bi[4];
        for (int d = 3; d >= 0; --d) {
            ii[d] = (int)(in % b[d]);
            in /= b[d];
            bi[d] = (int)(blk % nb[d]);
            blk /= nb[d];
        }
        double v[4];
        for (int d = 0; d < 4; ++d) {
            int node = bi[d] * b[d] + ii[d];
            v[d] = counts[d] == 1 ? centre[d]
                                  : centre[d] + half_width[d] * (2.0 * node / (double)(counts[d] - 1) - 1.0);
        }
        double *o = seeds + 6 * s;
        o[0] = vx;
        o[1] = vy;
        o[2] = v[0];
        o[3] = v[3] * cos(v[1]);
        o[4] = v[3] * sin(v[1]);
        o[5] = v[2];
    }
}

typedef struct {
    const or_field *f;
    const or_params *P;
    const double *seeds;
    const int8_t *charge;
    int64_t S;
    double *points;        /* propagate: [S][n_rec][6]; scan: NULL */
    int32_t *n_valid;
    const double *wires;
    int W;
    const int32_t *offs;
    const double *drift;
    const uint8_t *mask;
    double *rss;
    int32_t *n_in;
    double *dca_out;       /* [S][W] or NULL */
    int32_t *n_unconv;     /* [S] or NULL */
    int tid, nthreads;
} job_t;

static void *propagate_worker(void *arg)
{
    job_t *J = (job_t *)arg;
    int n_rec = oracle_n_rec(J->P);
    for (int64_t s = J->tid; s < J->S; s += J->nthreads)
        J->n_valid[s] = record_track(J->f, J->P, J->seeds + 6 * s, J->charge[s],
                                     J->points + (size_t)s * n_rec * 6);
    return NULL;
}

/* Unified per-seed RSS (the shape of Algorithm 3): record, then DCA for each wire in order. */
static void *scan_worker(void *arg)
{
    job_t *J = (job_t *)arg;
    int n_rec = oracle_n_rec(J->P);
    double *pts = (double *)malloc(sizeof(double) * 6 * (size_t)n_rec);
    for (int64_t s = J->tid; s < J->S; s += J->nthreads) {
        const double *sd = J->seeds + 6 * s;
        int q = J->charge[s];
        int nv = record_track(J->f, J->P, sd, q, pts);
        double P0 = sqrt(sd[3] * sd[3] + sd[4] * sd[4] + sd[5] * sd[5]);
        double rss = 0.0;
        int nin = 0, nunc = 0;
        for (int i = 0; i < J->W; ++i) {
            int any = 0;
            for (int j = J->offs[i]; j < J->offs[i + 1]; ++j)
                if (!J->mask[j]) any = 1;
            if (!any && !J->dca_out) continue;
            int conv;
            double D = dca_one(J->f, J->P, pts, nv, q, P0, J->wires + 6 * (size_t)i, &conv);
            if (J->dca_out) J->dca_out[(size_t)s * J->W + i] = D;
            if (!any) continue;
            if (!conv) ++nunc;
            double emin = INFINITY;
            for (int j = J->offs[i]; j < J->offs[i + 1]; ++j) {
                if (J->mask[j]) continue;
                double e = fabs(D - J->drift[j]);   /* min(d^L, d^R) for a hit at +-r (Eq. 1) */
                if (e < emin) emin = e;
            }
            double d = emin < J->P->lambda ? emin : J->P->lambda;
            if (emin < J->P->lambda) ++nin;
            rss += d * d;
        }
        J->rss[s] = rss;
        J->n_in[s] = nin;
        if (J->n_unconv) J->n_unconv[s] = nunc;
    }
    free(pts);
    return NULL;
}

static void run_threads(job_t *proto, int nthreads, void *(*fn)(void *))
{
    if (nthreads < 1) nthreads = 1;
    pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * nthreads);
    job_t *jobs = (job_t *)malloc(sizeof(job_t) * nthreads);
    for (int t = 0; t < nthreads; ++t) {
        jobs[t] = *proto;
        jobs[t].tid = t;
        jobs[t].nthreads = nthreads;
        pthread_create(&th[t], NULL, fn, &jobs[t]);
    }
    for (int t = 0; t < nthreads; ++t) pthread_join(th[t], NULL);
    free(th);
    free(jobs);
}

/* Track recording for S seeds; points [S][n_rec][6], n_valid [S]. */
void oracle_propagate(const or_field *f, const or_params *P, const double *seeds,
                      const int8_t *charge, int64_t S, double *points, int32_t *n_valid,
                      int nthreads)
{
    job_t J;
    memset(&J, 0, sizeof J);
    J.f = f;
    J.P = P;
    J.seeds = seeds;
    J.charge = charge;
    J.S = S;
    J.points = points;
    J.n_valid = n_valid;
    run_threads(&J, nthreads, propagate_worker);
}

/* RSS of every seed.  dca_out [S][W] (optional) receives every wire's DCA; n_unconv [S] (optional)
   counts wires with unmasked hits whose refinement did not converge. */
void oracle_scan(const or_field *f, const or_params *P, const double *seeds, const int8_t *charge,
                 int64_t S, const double *wires, int W, const int32_t *hit_offsets,
                 const double *drift, const uint8_t *mask, double *rss, int32_t *n_in,
                 double *dca_out, int32_t *n_unconv, int nthreads)
{
    job_t J;
    memset(&J, 0, sizeof J);
    J.f = f;
    J.P = P;
    J.seeds = seeds;
    J.charge = charge;
    J.S = S;
    J.wires = wires;
    J.W = W;
    J.offs = hit_offsets;
    J.drift = drift;
    J.mask = mask;
    J.rss = rss;
    J.n_in = n_in;
    J.dca_out = dca_out;
    J.n_unconv = n_unconv;
    run_threads(&J, nthreads, scan_worker);
}

/* ---------------------------------------------------------------------------------------------- */
/* Selection: the k seeds of lowest RSS, ascending; equal RSS ordered by seed index; NaN last.     */
/* ---------------------------------------------------------------------------------------------- */

typedef struct {
    double v;
    int64_t i;
} vi_t;

static int vi_cmp(const void *pa, const void *pb)
{
    const vi_t *a = (const vi_t *)pa, *b = (const vi_t *)pb;
    int an = isnan(a->v), bn = isnan(b->v);
    if (an != bn) return an - bn;
    if (!an && a->v < b->v) return -1;
    if (!an && a->v > b->v) return 1;
    return a->i < b->i ? -1 : (a->i > b->i ? 1 : 0);
}

void oracle_select(const double *rss, int64_t S, int k, int64_t *idx_out, double *rss_out)
{
    vi_t *a = (vi_t *)malloc(sizeof(vi_t) * (size_t)S);
    for (int64_t s = 0; s < S; ++s) {
        a[s].v = rss[s];
        a[s].i = s;
    }
    qsort(a, (size_t)S, sizeof(vi_t), vi_cmp);
    for (int j = 0; j < k && j < S; ++j) {
        idx_out[j] = a[j].i;
        rss_out[j] = a[j].v;
    }
    free(a);
}

/* ---------------------------------------------------------------------------------------------- */
/* Classification of one seed's hits (Sec. 2.1) and the mask of the next turn partition          */
/* ---------------------------------------------------------------------------------------------- */

void oracle_classify(const or_field *f, const or_params *P, const double seed[6], int q,
                     const double *wires, int W, const int32_t *hit_offsets, const double *drift,
                     uint8_t *mask, uint8_t *hit_class, double *dca_wire, int update_mask)
{
    int n_rec = oracle_n_rec(P);
    double *pts = (double *)malloc(sizeof(double) * 6 * (size_t)n_rec);
    int nv = record_track(f, P, seed, q, pts);
    double P0 = sqrt(seed[3] * seed[3] + seed[4] * seed[4] + seed[5] * seed[5]);
    int H = hit_offsets[W];
    for (int j = 0; j < H; ++j) hit_class[j] = 0;
    for (int i = 0; i < W; ++i) {
        int conv;
        double D = dca_one(f, P, pts, nv, q, P0, wires + 6 * (size_t)i, &conv);
        if (dca_wire) dca_wire[i] = D;
        int jbest = -1;
        double ebest = INFINITY;
        for (int j = hit_offsets[i]; j < hit_offsets[i + 1]; ++j) {
            if (mask[j]) continue;
            double e = fabs(D - drift[j]);
            if (e < ebest) {
                ebest = e;
                jbest = j;
            }
        }
        if (jbest >= 0 && ebest < P->lambda) hit_class[jbest] = 1;
    }
    if (update_mask)
        for (int j = 0; j < H; ++j) mask[j] |= hit_class[j];
    free(pts);
}

/* One RK4 step, exposed so the tests can check the integrator's order against the exact helix. */
void oracle_rk4_step(const or_field *f, int q, double P0, double y[6], double h)
{
    rk4_step(f, (double)q, P0, y, h);
}

void oracle_field_at(const or_field *f, const double x[3], double B[3]) { field_at(f, x, B); }
