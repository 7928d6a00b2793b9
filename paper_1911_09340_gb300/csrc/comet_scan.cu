// C ABI of the seed scan (declared and documented in include/comet_scan.h): argument validation on
// the host, the context's lazily allocated device scratch, and dispatch to the kernel launchers.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>

#include "comet_scan.h"
#include "internal.h"
#include "scan_ctx.h"

namespace comet {
namespace detail {

thread_local char g_err[512] = "";

comet_status fail(comet_status st, const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof g_err, fmt, ap);
    va_end(ap);
    return st;
}

comet_status cuda_fail(cudaError_t e, const char *where)
{
    return fail(COMET_ERR_CUDA, "%s: %s", where, cudaGetErrorString(e));
}

DeviceGuard::DeviceGuard(int dev)
{
    err = cudaGetDevice(&prev);
    if (err == cudaSuccess && prev != dev) err = cudaSetDevice(dev);
}

DeviceGuard::~DeviceGuard()
{
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
}

void BatchState::release()
{
    if (host) cudaFreeHost(host);
    if (dev) cudaFree(dev);
    if (copied) cudaEventDestroy(copied);
    host = dev = nullptr;
    copied = nullptr;
    recorded = ready = false;
    dtype = -1;
}

size_t esize(comet_dtype dt) { return dt == COMET_F32 ? sizeof(float) : sizeof(double); }

bool aligned(const void *p, size_t a) { return ((uintptr_t)p % a) == 0; }

comet_status check_dtype(comet_dtype dt)
{
    if (dt != COMET_F32 && dt != COMET_F64) return fail(COMET_ERR_INVALID_ARG, "dtype must be COMET_F32 or COMET_F64");
    return COMET_OK;
}

comet_status check_field(const comet_field *f)
{
    if (!f) return fail(COMET_ERR_INVALID_ARG, "field is NULL");
    if (f->kind == 0) {
        for (int i = 0; i < 3; ++i)
            if (!std::isfinite(f->b[i])) return fail(COMET_ERR_INVALID_ARG, "field.b must be finite");
        return COMET_OK;
    }
    if (f->kind != 1 && f->kind != 2)
        return fail(COMET_ERR_INVALID_ARG, "field.kind must be 0 (uniform), 1 (table) or 2 (interleaved table)");
    if (!f->table) return fail(COMET_ERR_INVALID_ARG, "field.table is NULL");
    if (!aligned(f->table, f->kind == 2 ? 16 : 4))
        return fail(COMET_ERR_INVALID_ARG, "field.table must be %d-byte aligned", f->kind == 2 ? 16 : 4);
    if (f->nx < 2 || f->ny < 2 || f->nz < 2) return fail(COMET_ERR_INVALID_ARG, "field table needs >= 2 nodes per axis");
    if (!(f->spacing > 0.0) || !std::isfinite(f->spacing)) return fail(COMET_ERR_INVALID_ARG, "field.spacing must be > 0");
    for (int i = 0; i < 3; ++i)
        if (!std::isfinite(f->origin[i])) return fail(COMET_ERR_INVALID_ARG, "field.origin must be finite");
    if ((double)f->nx * f->ny * f->nz * 3.0 > 9.0e18) return fail(COMET_ERR_INVALID_ARG, "field table too large");
    return COMET_OK;
}

comet_status check_params(const comet_scan_params *p, bool need_hits)
{
    if (!p) return fail(COMET_ERR_INVALID_ARG, "params is NULL");
    if (!(p->h > 0.0) || !std::isfinite(p->h)) return fail(COMET_ERR_INVALID_ARG, "params.h must be > 0");
    if (p->n_steps < 1) return fail(COMET_ERR_INVALID_ARG, "params.n_steps must be >= 1");
    if (p->stride < 1) return fail(COMET_ERR_INVALID_ARG, "params.stride must be >= 1");
    if (std::isnan(p->zmin) || std::isnan(p->zmax) || std::isnan(p->rmax))
        return fail(COMET_ERR_INVALID_ARG, "params target region must not be NaN");
    if (need_hits) {
        if (!(p->lambda > 0.0) || !std::isfinite(p->lambda)) return fail(COMET_ERR_INVALID_ARG, "params.lambda must be > 0");
        if (!(p->tol > 0.0) || !std::isfinite(p->tol)) return fail(COMET_ERR_INVALID_ARG, "params.tol must be > 0");
        if (p->max_iter < 0) return fail(COMET_ERR_INVALID_ARG, "params.max_iter must be >= 0");
    }
    return COMET_OK;
}

comet_status check_hits(comet_dtype dt, const void *wires, int32_t W, int32_t ldw,
                        const int32_t *offs, const void *drift, const void *mask)
{
    if (W < 0) return fail(COMET_ERR_INVALID_ARG, "W must be >= 0");
    if (W == 0) return COMET_OK;
    if (ldw < W) return fail(COMET_ERR_INVALID_ARG, "ldw must be >= W");
    if (!wires || !offs || !drift || !mask) return fail(COMET_ERR_INVALID_ARG, "wires, hit_offsets, drift and hit_mask are required when W > 0");
    if (!aligned(wires, esize(dt)) || !aligned(drift, esize(dt)) || !aligned(offs, 4))
        return fail(COMET_ERR_INVALID_ARG, "wires/drift/hit_offsets are misaligned for their element type");
    return COMET_OK;
}

int n_rec_of(const comet_scan_params *p) { return p->n_steps / p->stride + 1; }

// Segmentation and reaches of the closest-state search: identical for propagate (which writes the
// segment bounding spheres) and dca (which reads them).  Consecutive recorded states are at most
// stride*h apart along the track (|dx/ds| = |p|/P0 = 1 up to rounding); the margins cover the
// rounding of the distances in the working precision.  The refinement reaches up to h_rec beyond
// the first and the last recorded state, half an interval more than between states: R0 (and R1
// when segments hold several states) include that half interval; for one-state segments the DCA
// kernel adds it to its threshold where the state may be a track end.
SearchGeometry search_geometry(comet_dtype dtype, const comet_scan_params *p)
{
    SearchGeometry g;
    comet::dca_segments(n_rec_of(p), &g.G0, &g.G1);
    g.h_rec = p->h * p->stride;
    const double margin = dtype == COMET_F32 ? 4e-6 : 1e-9;
    g.half_rec = 0.5 * g.h_rec * (1.0 + 1e-4) + margin;
    g.R0 = (g.G0 / 2) * g.h_rec * (1.0 + 1e-4) + margin + g.half_rec;
    g.R1 = (g.G1 / 2) * g.h_rec * (1.0 + 1e-4) + margin + (g.G1 > 1 ? g.half_rec : 0.0);
    return g;
}

bool bounds_aligned(const void *b) { return b == nullptr || ((uintptr_t)b % 16) == 0; }

void fill_lat(const comet_lattice &lat, int8_t *charge_out, LatArgs *a)
{
    a->vx = lat.vx;
    a->vy = lat.vy;
    for (int d = 0; d < 4; ++d) {
        a->centre[d] = lat.centre[d];
        a->half_width[d] = lat.half_width[d];
        a->counts[d] = lat.counts[d];
    }
    a->charge = lat.charge;
    a->charge_out = charge_out;
}

// Node i of n of one lattice dimension: centre + half_width (2 i / (n - 1) - 1), each operation
// rounded on its own (no fused multiply-add), the same arithmetic as the oracle's lattice.
static double host_lattice_node(double centre, double half_width, int n, int i)
{
    if (n == 1) return centre;
    volatile double q = (2.0 * i) / (double)(n - 1);
    volatile double t = q - 1.0;
    volatile double u = half_width * t;
    return centre + u;
}

void fill_lat_table(const LatArgs &a, LatTable *t)
{
    t->use = 0;
    int tot = 0;
    for (int d = 0; d < 4; ++d) tot += a.counts[d];
    if (tot > kLatParamNodes || a.counts[1] > kLatParamPhi) return;
    int o = 0;
    for (int d = 0; d < 4; ++d) {
        for (int k = 0; k < a.counts[d]; ++k)
            t->node[o + k] = host_lattice_node(a.centre[d], a.half_width[d], a.counts[d], k);
        o += a.counts[d];
    }
    for (int k = 0; k < a.counts[1]; ++k) {
        const double v = t->node[a.counts[0] + k];
        t->cphi[k] = std::cos(v);
        t->sphi[k] = std::sin(v);
    }
    t->use = 1;
}

void fill_prop(comet_dtype, const comet_scan_params *p, const SearchGeometry &sg, const void *seeds,
               const int8_t *charge, int64_t S, void *points, int32_t *n_valid, void *bounds, PropArgs *a)
{
    a->bounds = bounds;
    a->G0 = sg.G0;
    a->G1 = sg.G1;
    a->R0 = sg.R0;
    a->R1 = sg.R1;
    a->seeds = seeds;
    a->charge = charge;
    a->S = S;
    a->points = points;
    a->n_valid = n_valid;
    a->h = p->h;
    a->zmin = p->zmin;
    a->zmax = p->zmax;
    a->rmax = p->rmax;
    a->n_steps = p->n_steps;
    a->stride = p->stride;
    a->h_ff.hi = (float)p->h;
    a->h_ff.lo = (float)(p->h - (double)a->h_ff.hi);
    a->lim_f[0] = (float)p->zmin;
    a->lim_f[1] = (float)p->zmax;
    a->lim_f[2] = (float)(p->rmax * p->rmax);
    a->lim_f[3] = (float)sg.R0;
    a->lim_f[4] = (float)sg.R1;
    a->n_rec = n_rec_of(p);
}

void fill_dca(comet_ctx *ctx, comet_dtype dtype, const comet_scan_params *p, const SearchGeometry &sg,
              const void *points, const int32_t *n_valid, const int8_t *charge, int64_t S,
              const void *bounds, const void *wires, int32_t W, int32_t ldw, const int32_t *offs,
              const void *drift, const uint8_t *mask, void *rss, int32_t *n_in, void *dca_out,
              int32_t *n_unconverged, DcaArgs *a)
{
    a->points = points;
    a->n_valid = n_valid;
    a->charge = charge;
    a->S = S;
    a->n_rec = n_rec_of(p);
    a->wires = wires;
    a->W = W;
    a->ldw = W > 0 ? ldw : 0;
    a->offs = offs;
    a->drift = drift;
    a->mask = mask;
    a->rss = rss;
    a->n_in = n_in;
    a->dca_out = W > 0 ? dca_out : nullptr;
    a->n_unconv = n_unconverged;
    a->status = ctx->status;
    a->counter = ctx->status + 16;
    a->wait_ns = ctx->copy_wait_ns;
    a->max_ctas_per_sm = ctx->dca_ctas_per_sm;
    a->batch_groups = 0;
    a->best_idx_out = nullptr;
    a->best_rss_out = nullptr;
    a->best_slots = nullptr;
    a->best_slots_cap = 0;
    a->best_counter = nullptr;
    a->lambda = p->lambda;
    a->tol = p->tol;
    a->max_iter = p->max_iter;
    a->G0 = sg.G0;
    a->G1 = sg.G1;
    a->R0 = sg.R0;
    a->R1 = sg.R1;
    a->half_rec = sg.half_rec;
    a->h_rec = sg.h_rec;
    a->lambda_f = (float)a->lambda;
    a->tol_f = (float)a->tol;
    a->half_rec_f = (float)a->half_rec;
    a->h_rec_f = (float)a->h_rec;
    a->margin = dtype == COMET_F32 ? 4e-6 : 1e-9;
    a->margin_f = (float)a->margin;
    a->bounds = bounds;
    a->exact_all = dca_out != nullptr;
    a->n_chunks = comet::dca_wire_chunks(W, S, ctx->dca_chunk_wires);
    a->part = nullptr;
    a->arrive = nullptr;
}

void fill_cls(comet_ctx *ctx, comet_dtype, const comet_scan_params *p, const void *points,
              const int32_t *n_valid, const int8_t *charge, int64_t S, const int64_t *seed_index,
              const void *wires, int32_t W, int32_t ldw, const int32_t *offs, const void *drift,
              uint8_t *mask, uint8_t *hit_class, void *dca_wire, int32_t update_mask, ClsArgs *a)
{
    a->points = points;
    a->n_valid = n_valid;
    a->charge = charge;
    a->S = S;
    a->n_rec = n_rec_of(p);
    a->seed_index = seed_index;
    a->wires = wires;
    a->W = W;
    a->ldw = ldw;
    a->offs = offs;
    a->drift = drift;
    a->mask = mask;
    a->hit_class = hit_class;
    a->dca_wire = dca_wire;
    a->status = ctx->status;
    a->lambda = p->lambda;
    a->tol = p->tol;
    a->h_rec = p->h * p->stride;
    a->max_iter = p->max_iter;
    a->update_mask = update_mask;
}

} // namespace detail
} // namespace comet

using namespace comet::detail;
#define CHECK(expr) COMET_CHECK(expr)

extern "C" {

const char *comet_last_error(void) { return g_err; }

comet_status comet_ctx_create(int device, comet_ctx **out)
{
    if (!out) return fail(COMET_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    int n = 0;
    cudaError_t e = cudaGetDeviceCount(&n);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDeviceCount");
    if (device < 0 || device >= n) return fail(COMET_ERR_INVALID_ARG, "device %d out of range (%d devices)", device, n);
    DeviceGuard g(device);
    if (g.err != cudaSuccess) return cuda_fail(g.err, "cudaSetDevice");
    comet_ctx *c = new (std::nothrow) comet_ctx;
    if (!c) return fail(COMET_ERR_NO_MEMORY, "host allocation failed");
    c->device = device;
    e = cudaMalloc(&c->status, 256);
    if (e != cudaSuccess) {
        delete c;
        return e == cudaErrorMemoryAllocation ? fail(COMET_ERR_NO_MEMORY, "cudaMalloc(status)") : cuda_fail(e, "cudaMalloc(status)");
    }
    e = cudaMemset(c->status, 0, 256);
    if (e != cudaSuccess) {
        cudaFree(c->status);
        delete c;
        return cuda_fail(e, "cudaMemset(status)");
    }
    *out = c;
    return COMET_OK;
}

void comet_ctx_destroy(comet_ctx *ctx)
{
    if (!ctx) return;
    {
        DeviceGuard g(ctx->device);
        cudaDeviceSynchronize();
        if (ctx->scratch) cudaFree(ctx->scratch);
        if (ctx->status) cudaFree(ctx->status);
        if (ctx->dca_part) cudaFree(ctx->dca_part);
        if (ctx->dca_arrive) cudaFree(ctx->dca_arrive);
        if (ctx->dca_best) cudaFree(ctx->dca_best);
        ctx->batch.release();
        cudaGetLastError();   // destroy reports nothing: leave no error behind for the next call
    }
    delete ctx;
}

comet_status comet_ctx_status(comet_ctx *ctx, int32_t *flags)
{
    if (!ctx || !flags) return fail(COMET_ERR_INVALID_ARG, "ctx and flags are required");
    DeviceGuard g(ctx->device);
    if (g.err != cudaSuccess) return cuda_fail(g.err, "cudaSetDevice");
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceSynchronize");
    e = cudaMemcpy(flags, ctx->status, sizeof(int32_t), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpy(status)");
    return COMET_OK;
}

comet_status comet_ctx_set_copy_wait(comet_ctx *ctx, int64_t ns)
{
    if (!ctx) return fail(COMET_ERR_INVALID_ARG, "ctx is NULL");
    if (ns < 0) return fail(COMET_ERR_INVALID_ARG, "the copy wait limit must be >= 0 ns");
    ctx->copy_wait_ns = (uint64_t)ns;
    return COMET_OK;
}

comet_status comet_ctx_set_dca_ctas_per_sm(comet_ctx *ctx, int32_t n)
{
    if (!ctx) return fail(COMET_ERR_INVALID_ARG, "ctx is NULL");
    if (n < 0 || n > 64) return fail(COMET_ERR_INVALID_ARG, "CTAs per SM must be in 0 .. 64");
    ctx->dca_ctas_per_sm = n;
    return COMET_OK;
}

comet_status comet_ctx_set_dca_chunk_wires(comet_ctx *ctx, int32_t wires)
{
    if (!ctx) return fail(COMET_ERR_INVALID_ARG, "ctx is NULL");
    if (wires != 0 && (wires < 4 || wires > 1024))
        return fail(COMET_ERR_INVALID_ARG, "wires per chunk must be 0 (automatic) or in 4 .. 1024");
    ctx->dca_chunk_wires = wires;
    return COMET_OK;
}

comet_status comet_ctx_set_record_blocks(comet_ctx *ctx, int32_t on)
{
    if (!ctx) return fail(COMET_ERR_INVALID_ARG, "ctx is NULL");
    if (on != 0 && on != 1) return fail(COMET_ERR_INVALID_ARG, "record_blocks must be 0 or 1");
    ctx->record_blocks = on;
    return COMET_OK;
}

comet_status comet_kernel_arch(int32_t *sm_version)
{
    if (!sm_version) return fail(COMET_ERR_INVALID_ARG, "sm_version is NULL");
    int v = 0;
    cudaError_t e = comet::kernel_binary_version(&v);
    if (e != cudaSuccess) return cuda_fail(e, "cudaFuncGetAttributes");
    *sm_version = v;
    return COMET_OK;
}

comet_status comet_scan_lattice(comet_ctx *ctx, comet_dtype dtype, const comet_lattice *lat,
                                void *seeds, int8_t *charge_out, int64_t S, comet_stream stream)
{
    if (!ctx) return fail(COMET_ERR_INVALID_ARG, "ctx is NULL");
    CHECK(check_dtype(dtype));
    if (!lat) return fail(COMET_ERR_INVALID_ARG, "lattice is NULL");
    int64_t prod = 1;
    for (int d = 0; d < 4; ++d) {
        if (lat->counts[d] < 1) return fail(COMET_ERR_INVALID_ARG, "lattice.counts must be >= 1");
        prod *= lat->counts[d];
        if (prod > (int64_t)1 << 40) return fail(COMET_ERR_INVALID_ARG, "lattice too large");
        if (!std::isfinite(lat->centre[d]) || !std::isfinite(lat->half_width[d]))
            return fail(COMET_ERR_INVALID_ARG, "lattice centre/half_width must be finite");
    }
    if (S != prod) return fail(COMET_ERR_INVALID_ARG, "S (%lld) != product of lattice counts (%lld)", (long long)S, (long long)prod);
    if (!seeds || !aligned(seeds, esize(dtype))) return fail(COMET_ERR_INVALID_ARG, "seeds is NULL or misaligned");
    if (lat->charge < -128 || lat->charge > 127) return fail(COMET_ERR_INVALID_ARG, "lattice.charge must fit int8");
    DeviceGuard g(ctx->device);
    if (g.err != cudaSuccess) return cuda_fail(g.err, "cudaSetDevice");
    comet::LatArgs a;
    fill_lat(*lat, charge_out, &a);
    comet::LatTable t;
    fill_lat_table(a, &t);
    cudaError_t e = comet::launch_lattice(dtype, a, t, seeds, S, (cudaStream_t)stream);
    return e == cudaSuccess ? COMET_OK : cuda_fail(e, "lattice launch");
}

comet_status comet_scan_refine_refs(comet_ctx *ctx, comet_dtype dtype, const void *seeds, int64_t S,
                                    const int64_t *idx, int32_t M, const double half_width[4],
                                    int32_t K, double *refs_out, int32_t *n_refs_out,
                                    comet_stream stream)
{
    if (!ctx) return fail(COMET_ERR_INVALID_ARG, "ctx is NULL");
    CHECK(check_dtype(dtype));
    if (S <= 0) return fail(COMET_ERR_INVALID_ARG, "S must be > 0");
    if (!seeds || !aligned(seeds, esize(dtype))) return fail(COMET_ERR_INVALID_ARG, "seeds is NULL or misaligned");
    if (!idx || !aligned(idx, 8)) return fail(COMET_ERR_INVALID_ARG, "idx is NULL or misaligned");
    if (M < 1 || M > (1 << 20)) return fail(COMET_ERR_INVALID_ARG, "M must be in 1 .. 1048576");
    if (K < 1 || K > 32) return fail(COMET_ERR_INVALID_ARG, "K must be in 1 .. 32");
    if (!half_width) return fail(COMET_ERR_INVALID_ARG, "half_width is NULL");
    for (int d = 0; d < 4; ++d)
        if (!std::isfinite(half_width[d]) || half_width[d] < 0.0)
            return fail(COMET_ERR_INVALID_ARG, "half_width must be finite and >= 0");
    if (!refs_out || !aligned(refs_out, 8)) return fail(COMET_ERR_INVALID_ARG, "refs_out is NULL or misaligned");
    if (!n_refs_out || !aligned(n_refs_out, 4)) return fail(COMET_ERR_INVALID_ARG, "n_refs_out is NULL or misaligned");
    DeviceGuard g(ctx->device);
    if (g.err != cudaSuccess) return cuda_fail(g.err, "cudaSetDevice");
    comet::RefArgs a;
    a.seeds = seeds;
    a.S = S;
    a.idx = idx;
    a.M = M;
    a.K = K;
    for (int d = 0; d < 4; ++d) a.half_width[d] = half_width[d];
    a.refs_out = refs_out;
    a.n_refs_out = n_refs_out;
    cudaError_t e = comet::launch_refine_refs(dtype, a, (cudaStream_t)stream);
    return e == cudaSuccess ? COMET_OK : cuda_fail(e, "refine_refs launch");
}

comet_status comet_scan_lattice_refined(comet_ctx *ctx, comet_dtype dtype, const comet_lattice *shape,
                                        const double *refs, const int32_t *n_refs, int32_t K,
                                        void *seeds, int8_t *charge_out, int64_t S,
                                        comet_stream stream)
{
    if (!ctx) return fail(COMET_ERR_INVALID_ARG, "ctx is NULL");
    CHECK(check_dtype(dtype));
    if (!shape) return fail(COMET_ERR_INVALID_ARG, "shape is NULL");
    if (K < 1 || K > 32) return fail(COMET_ERR_INVALID_ARG, "K must be in 1 .. 32");
    int64_t prod = 1;
    for (int d = 0; d < 4; ++d) {
        if (shape->counts[d] < 1) return fail(COMET_ERR_INVALID_ARG, "shape.counts must be >= 1");
        prod *= shape->counts[d];
        if (prod > (int64_t)1 << 36) return fail(COMET_ERR_INVALID_ARG, "lattice too large");
        if (!std::isfinite(shape->half_width[d]))
            return fail(COMET_ERR_INVALID_ARG, "shape.half_width must be finite");
    }
    if (S != prod * K) return fail(COMET_ERR_INVALID_ARG, "S (%lld) != K x product of shape counts (%lld)", (long long)S, (long long)(prod * K));
    if (!refs || !aligned(refs, 8)) return fail(COMET_ERR_INVALID_ARG, "refs is NULL or misaligned");
    if (!n_refs || !aligned(n_refs, 4)) return fail(COMET_ERR_INVALID_ARG, "n_refs is NULL or misaligned");
    if (!seeds || !aligned(seeds, esize(dtype))) return fail(COMET_ERR_INVALID_ARG, "seeds is NULL or misaligned");
    if (shape->charge < -128 || shape->charge > 127) return fail(COMET_ERR_INVALID_ARG, "shape.charge must fit int8");
    DeviceGuard g(ctx->device);
    if (g.err != cudaSuccess) return cuda_fail(g.err, "cudaSetDevice");
    comet::LatArgs a;
    a.vx = shape->vx;
    a.vy = shape->vy;
    for (int d = 0; d < 4; ++d) {
        a.centre[d] = 0.0;
        a.half_width[d] = shape->half_width[d];
        a.counts[d] = shape->counts[d];
    }
    a.charge = shape->charge;
    a.charge_out = charge_out;
    cudaError_t e = comet::launch_lattice_refined(dtype, a, refs, n_refs, K, seeds, S, (cudaStream_t)stream);
    return e == cudaSuccess ? COMET_OK : cuda_fail(e, "lattice_refined launch");
}

comet_status comet_scan_jacobian(comet_ctx *ctx, comet_dtype dtype, const comet_field *field,
                                 const comet_scan_params *params, const double *theta, int64_t S,
                                 double vx, double vy, int32_t charge, const void *wires, int32_t W,
                                 int32_t ldw, const int32_t *hit_offsets, const void *drift,
                                 const uint8_t *hit_mask, double tau, double *work,
                                 double *srss_out, double *grad_out, double *jtj_out,
                                 double *jtr_out, double *dca_out, double *jac_out,
                                 double *grad6_out, int32_t *n_unconverged, comet_stream stream)
{
    if (!ctx) return fail(COMET_ERR_INVALID_ARG, "ctx is NULL");
    CHECK(check_dtype(dtype));
    if (dtype != COMET_F64) return fail(COMET_ERR_UNSUPPORTED, "comet_scan_jacobian needs COMET_F64");
    CHECK(check_field(field));
    if (field->kind != 0 || field->b[0] != 0.0 || field->b[1] != 0.0)
        return fail(COMET_ERR_UNSUPPORTED, "comet_scan_jacobian needs a uniform field along z");
    CHECK(check_params(params, true));
    if (S <= 0 || S > ((int64_t)1 << 24)) return fail(COMET_ERR_INVALID_ARG, "S must be in 1 .. 2^24");
    if (W < 0 || ldw < W) return fail(COMET_ERR_INVALID_ARG, "need 0 <= W <= ldw");
    if (!(tau > 0.0) || !std::isfinite(tau)) return fail(COMET_ERR_INVALID_ARG, "tau must be > 0");
    if (!std::isfinite(vx) || !std::isfinite(vy)) return fail(COMET_ERR_INVALID_ARG, "vertex must be finite");
    const void *req[] = {theta, work, srss_out, grad_out, jtj_out, jtr_out};
    for (const void *q : req)
        if (!q || !aligned(q, 8)) return fail(COMET_ERR_INVALID_ARG, "a required array is NULL or misaligned");
    if (W > 0 && (!wires || !hit_offsets || !drift || !hit_mask || !aligned(wires, 8) || !aligned(drift, 8) ||
                  !aligned(hit_offsets, 4)))
        return fail(COMET_ERR_INVALID_ARG, "wires / hits NULL or misaligned");
    if ((dca_out && !aligned(dca_out, 8)) || (jac_out && !aligned(jac_out, 8)) ||
        (grad6_out && !aligned(grad6_out, 8)))
        return fail(COMET_ERR_INVALID_ARG, "dca_out / jac_out / grad6_out misaligned");
    if (charge < -128 || charge > 127) return fail(COMET_ERR_INVALID_ARG, "charge must fit int8");
    DeviceGuard g(ctx->device);
    if (g.err != cudaSuccess) return cuda_fail(g.err, "cudaSetDevice");
    comet::JacArgs a;
    a.theta = theta;
    a.S = S;
    a.vx = vx;
    a.vy = vy;
    a.bz = field->b[2];
    a.charge = charge;
    a.h = params->h;
    a.stride = params->stride;
    a.n_rec = n_rec_of(params);
    a.h_rec = params->h * params->stride;
    a.zmin = params->zmin;
    a.zmax = params->zmax;
    a.rmax2 = params->rmax * params->rmax;
    a.tol = params->tol;
    a.max_iter = params->max_iter;
    a.lambda = params->lambda;
    a.tau = tau;
    a.wires = wires;
    a.W = W;
    a.ldw = ldw;
    a.offs = hit_offsets;
    a.drift = (const double *)drift;
    a.mask = hit_mask;
    a.work = work;
    a.srss_out = srss_out;
    a.grad_out = grad_out;
    a.jtj_out = jtj_out;
    a.jtr_out = jtr_out;
    a.dca_out = dca_out;
    a.jac_out = jac_out;
    a.grad6_out = grad6_out;
    a.n_unconv = n_unconverged;
    cudaError_t e = comet::launch_jacobian(a, (cudaStream_t)stream);
    return e == cudaSuccess ? COMET_OK : cuda_fail(e, "jacobian launch");
}

comet_status comet_scan_gn_step(comet_ctx *ctx, double *theta, int64_t S, const double *jtj,
                                const double *jtr, double mu, comet_stream stream)
{
    if (!ctx) return fail(COMET_ERR_INVALID_ARG, "ctx is NULL");
    if (S <= 0 || S > ((int64_t)1 << 24)) return fail(COMET_ERR_INVALID_ARG, "S must be in 1 .. 2^24");
    if (!theta || !jtj || !jtr || !aligned(theta, 8) || !aligned(jtj, 8) || !aligned(jtr, 8))
        return fail(COMET_ERR_INVALID_ARG, "theta / jtj / jtr NULL or misaligned");
    if (!(mu >= 0.0) || !std::isfinite(mu)) return fail(COMET_ERR_INVALID_ARG, "mu must be >= 0");
    DeviceGuard g(ctx->device);
    if (g.err != cudaSuccess) return cuda_fail(g.err, "cudaSetDevice");
    cudaError_t e = comet::launch_gn_step(theta, S, jtj, jtr, mu, (cudaStream_t)stream);
    return e == cudaSuccess ? COMET_OK : cuda_fail(e, "gn_step launch");
}

comet_status comet_scan_lm_step(comet_ctx *ctx, int64_t S, double *theta, double *srss, double *jtj,
                                double *jtr, double *theta_try, const double *srss_try,
                                const double *jtj_try, const double *jtr_try, double *mu, double up,
                                double down, int32_t first, comet_stream stream)
{
    if (!ctx) return fail(COMET_ERR_INVALID_ARG, "ctx is NULL");
    if (S <= 0 || S > ((int64_t)1 << 24)) return fail(COMET_ERR_INVALID_ARG, "S must be in 1 .. 2^24");
    const void *req[] = {theta, srss, jtj, jtr, theta_try, mu};
    for (const void *q : req)
        if (!q || !aligned(q, 8)) return fail(COMET_ERR_INVALID_ARG, "a required array is NULL or misaligned");
    if (!first) {
        const void *tr[] = {srss_try, jtj_try, jtr_try};
        for (const void *q : tr)
            if (!q || !aligned(q, 8)) return fail(COMET_ERR_INVALID_ARG, "the trial's arrays are NULL or misaligned");
    }
    if (!(up >= 1.0) || !std::isfinite(up) || !(down > 0.0) || !(down <= 1.0))
        return fail(COMET_ERR_INVALID_ARG, "need up >= 1 and 0 < down <= 1");
    DeviceGuard g(ctx->device);
    if (g.err != cudaSuccess) return cuda_fail(g.err, "cudaSetDevice");
    comet::LmArgs a;
    a.S = S;
    a.theta = theta;
    a.srss = srss;
    a.jtj = jtj;
    a.jtr = jtr;
    a.theta_try = theta_try;
    a.srss_try = srss_try;
    a.jtj_try = jtj_try;
    a.jtr_try = jtr_try;
    a.mu = mu;
    a.up = up;
    a.down = down;
    a.mu_min = 1e-12;
    a.mu_max = 1e12;
    a.first = first != 0;
    cudaError_t e = comet::launch_lm_step(a, (cudaStream_t)stream);
    return e == cudaSuccess ? COMET_OK : cuda_fail(e, "lm_step launch");
}

comet_status comet_scan_propagate(comet_ctx *ctx, comet_dtype dtype, const comet_field *field,
                                  const comet_scan_params *params, const void *seeds,
                                  const int8_t *charge, int64_t S, void *points, int32_t *n_valid,
                                  void *bounds, comet_stream stream)
{
    if (!ctx) return fail(COMET_ERR_INVALID_ARG, "ctx is NULL");
    CHECK(check_dtype(dtype));
    CHECK(check_field(field));
    CHECK(check_params(params, false));
    if (S < 0) return fail(COMET_ERR_INVALID_ARG, "S must be >= 0");
    if (S == 0) return COMET_OK;
    if (!seeds || !charge || !points || !n_valid) return fail(COMET_ERR_INVALID_ARG, "seeds, charge, points and n_valid are required");
    if (!aligned(seeds, esize(dtype)) || !aligned(points, esize(dtype)) || !aligned(n_valid, 4) ||
        !bounds_aligned(bounds))
        return fail(COMET_ERR_INVALID_ARG, "seeds/points/n_valid/bounds misaligned for their element type");
    DeviceGuard g(ctx->device);
    if (g.err != cudaSuccess) return cuda_fail(g.err, "cudaSetDevice");
    const SearchGeometry sg = search_geometry(dtype, params);
    comet::PropArgs a;
    fill_prop(dtype, params, sg, seeds, charge, S, points, n_valid, bounds, &a);
    cudaError_t e = comet::launch_propagate(dtype, *field, a, ctx->record_blocks != 0, (cudaStream_t)stream);
    return e == cudaSuccess ? COMET_OK : cuda_fail(e, "propagate launch");
}

comet_status comet_scan_dca(comet_ctx *ctx, comet_dtype dtype, const comet_field *field,
                            const comet_scan_params *params, const void *points,
                            const int32_t *n_valid, const int8_t *charge, int64_t S,
                            const void *bounds, const void *wires, int32_t W, int32_t ldw, const int32_t *hit_offsets,
                            const void *drift, const uint8_t *hit_mask, void *rss, int32_t *n_in,
                            void *dca_out, int32_t *n_unconverged, int64_t *best_idx_out,
                            void *best_rss_out, comet_stream stream)
{
    if (!ctx) return fail(COMET_ERR_INVALID_ARG, "ctx is NULL");
    CHECK(check_dtype(dtype));
    CHECK(check_field(field));
    CHECK(check_params(params, true));
    if (S < 0) return fail(COMET_ERR_INVALID_ARG, "S must be >= 0");
    CHECK(check_hits(dtype, wires, W, ldw, hit_offsets, drift, hit_mask));
    if (S == 0) return COMET_OK;
    if (!points || !n_valid || !charge || !rss || !n_in) return fail(COMET_ERR_INVALID_ARG, "points, n_valid, charge, rss and n_in are required");
    if (!aligned(points, esize(dtype)) || !aligned(rss, esize(dtype)) || !aligned(n_valid, 4) ||
        !aligned(n_in, 4) || (dca_out && !aligned(dca_out, esize(dtype))) ||
        (n_unconverged && !aligned(n_unconverged, 4)) || !bounds_aligned(bounds) ||
        (best_idx_out && !aligned(best_idx_out, 8)) || (best_rss_out && !aligned(best_rss_out, esize(dtype))))
        return fail(COMET_ERR_INVALID_ARG, "an array is misaligned for its element type");
    if (best_rss_out && !best_idx_out) return fail(COMET_ERR_INVALID_ARG, "best_rss_out needs best_idx_out");
    DeviceGuard g(ctx->device);
    if (g.err != cudaSuccess) return cuda_fail(g.err, "cudaSetDevice");
    comet::DcaArgs a;
    fill_dca(ctx, dtype, params, search_geometry(dtype, params), points, n_valid, charge, S, bounds, wires,
             W, ldw, hit_offsets, drift, hit_mask, rss, n_in, dca_out, n_unconverged, &a);
    if (a.n_chunks > 1) {
        // per-chunk partial sums and per-group arrival counters, grown on demand; the counters are
        // zeroed once here and left zero by every launch
        // sized at first for the chunks of max(W, 256) wires, so that events of up to 256 wires
        // never reallocate
        const int nc_alloc = comet::dca_wire_chunks(W > 256 ? W : 256, S, ctx->dca_chunk_wires);
        const size_t need = (size_t)(a.n_chunks > nc_alloc ? a.n_chunks : nc_alloc) * (size_t)S * (2 * esize(dtype) + 4);
        const size_t groups = (size_t)((S + 31) / 32);
        if (need > ctx->dca_part_bytes) {
            // grown at least twofold, so that calls with more wires or seeds rarely reallocate
            const size_t want = need > 2 * ctx->dca_part_bytes ? need : 2 * ctx->dca_part_bytes;
            if (ctx->dca_part) cudaFree(ctx->dca_part);
            ctx->dca_part = nullptr;
            ctx->dca_part_bytes = 0;
            cudaError_t e = cudaMalloc(&ctx->dca_part, want);
            if (e != cudaSuccess)
                return e == cudaErrorMemoryAllocation ? fail(COMET_ERR_NO_MEMORY, "cudaMalloc(dca partial sums, %zu B)", want) : cuda_fail(e, "cudaMalloc");
            ctx->dca_part_bytes = want;
        }
        if (groups > ctx->dca_arrive_n) {
            const size_t n = groups > 2 * ctx->dca_arrive_n ? groups : 2 * ctx->dca_arrive_n;
            if (ctx->dca_arrive) cudaFree(ctx->dca_arrive);
            ctx->dca_arrive = nullptr;
            ctx->dca_arrive_n = 0;
            cudaError_t e = cudaMalloc(&ctx->dca_arrive, n * 4);
            if (e != cudaSuccess)
                return e == cudaErrorMemoryAllocation ? fail(COMET_ERR_NO_MEMORY, "cudaMalloc(dca counters, %zu B)", n * 4) : cuda_fail(e, "cudaMalloc");
            e = cudaMemsetAsync(ctx->dca_arrive, 0, n * 4, (cudaStream_t)stream);
            if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync");
            ctx->dca_arrive_n = n;
        }
        a.part = ctx->dca_part;
        a.arrive = ctx->dca_arrive;
    }
    if (best_idx_out) {
        // one slot per CTA: the persistent grid is at most 64 CTAs per SM, the tiled one S / 128
        const int64_t cap_p = (int64_t)64 * comet::device_sm_count();
        const int64_t cap_t = (S + 127) / 128;
        const int64_t cap = cap_p > cap_t ? cap_p : cap_t;
        if (cap > ctx->dca_best_cap) {
            if (ctx->dca_best) cudaFree(ctx->dca_best);
            ctx->dca_best = nullptr;
            ctx->dca_best_cap = 0;
            cudaError_t e = cudaMalloc(&ctx->dca_best, (size_t)cap * 16);
            if (e != cudaSuccess)
                return e == cudaErrorMemoryAllocation ? fail(COMET_ERR_NO_MEMORY, "cudaMalloc(dca selection slots)") : cuda_fail(e, "cudaMalloc");
            ctx->dca_best_cap = cap;
        }
        a.best_idx_out = best_idx_out;
        a.best_rss_out = best_rss_out;
        a.best_slots = ctx->dca_best;
        a.best_slots_cap = ctx->dca_best_cap;
        a.best_counter = (uint32_t *)(ctx->status + 20);
    }
    cudaError_t e = comet::launch_dca(dtype, *field, a, (cudaStream_t)stream);
    return e == cudaSuccess ? COMET_OK : cuda_fail(e, "dca launch");
}

comet_status comet_scan_select(comet_ctx *ctx, comet_dtype dtype, const void *rss, int64_t S,
                               int32_t k, int64_t *idx_out, void *rss_out, comet_stream stream)
{
    if (!ctx) return fail(COMET_ERR_INVALID_ARG, "ctx is NULL");
    CHECK(check_dtype(dtype));
    if (S < 1) return fail(COMET_ERR_INVALID_ARG, "S must be >= 1");
    if (k < 1 || k > 64 || k > S) return fail(COMET_ERR_INVALID_ARG, "k must be in [1, min(64, S)]");
    if (!rss || !idx_out) return fail(COMET_ERR_INVALID_ARG, "rss and idx_out are required");
    if (!aligned(rss, esize(dtype)) || !aligned(idx_out, 8) || (rss_out && !aligned(rss_out, esize(dtype))))
        return fail(COMET_ERR_INVALID_ARG, "an array is misaligned for its element type");
    DeviceGuard g(ctx->device);
    if (g.err != cudaSuccess) return cuda_fail(g.err, "cudaSetDevice");
    comet::SelArgs a;
    a.rss = rss;
    a.S = S;
    a.k = k;
    a.idx_out = idx_out;
    a.rss_out = rss_out;
    const size_t need = comet::select_scratch_bytes(dtype, S, k, &a.n_blocks);
    if (need > ctx->scratch_bytes) {
        // grow: the old buffer may still be in use by queued work on any stream
        cudaError_t e = cudaDeviceSynchronize();
        if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceSynchronize");
        if (ctx->scratch) cudaFree(ctx->scratch);
        ctx->scratch = nullptr;
        ctx->scratch_bytes = 0;
        size_t want = need < ((size_t)1 << 20) ? ((size_t)1 << 20) : need;
        e = cudaMalloc(&ctx->scratch, want);
        if (e != cudaSuccess)
            return e == cudaErrorMemoryAllocation ? fail(COMET_ERR_NO_MEMORY, "cudaMalloc(select scratch, %zu B)", want) : cuda_fail(e, "cudaMalloc");
        ctx->scratch_bytes = want;
    }
    a.scratch = ctx->scratch;
    cudaError_t e = comet::launch_select(dtype, a, (cudaStream_t)stream);
    return e == cudaSuccess ? COMET_OK : cuda_fail(e, "select launch");
}

comet_status comet_scan_select_noalloc(comet_dtype dtype, const void *rss, int64_t S, int32_t k,
                                       int64_t *idx_out, void *rss_out, comet_stream stream)
{
    CHECK(check_dtype(dtype));
    if (S < 1) return fail(COMET_ERR_INVALID_ARG, "S must be >= 1");
    if (k < 1 || k > 64 || k > S) return fail(COMET_ERR_INVALID_ARG, "k must be in [1, min(64, S)]");
    if (!rss || !idx_out) return fail(COMET_ERR_INVALID_ARG, "rss and idx_out are required");
    if (!aligned(rss, esize(dtype)) || !aligned(idx_out, 8) || (rss_out && !aligned(rss_out, esize(dtype))))
        return fail(COMET_ERR_INVALID_ARG, "an array is misaligned for its element type");
    // the arrays must live on the current device, where the kernels and the scratch are
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    const void *arrays[3] = {rss, idx_out, rss_out};
    for (const void *q : arrays) {
        if (!q) continue;
        cudaPointerAttributes at;
        e = cudaPointerGetAttributes(&at, q);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(COMET_ERR_INVALID_ARG, "rss / idx_out / rss_out is not a device pointer");
        }
        if ((at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged) || at.device != dev)
            return fail(COMET_ERR_INVALID_ARG,
                        "rss / idx_out / rss_out must be device memory of the current device (%d)", dev);
    }
    comet::SelArgs a;
    a.rss = rss;
    a.S = S;
    a.k = k;
    a.idx_out = idx_out;
    a.rss_out = rss_out;
    const size_t need = comet::select_scratch_bytes(dtype, S, k, &a.n_blocks);
    if (need > comet::kStaticSelectScratchBytes)
        return fail(COMET_ERR_INVALID_ARG,
                    "S = %lld with k = %d needs %zu bytes of scratch; the static scratch holds %zu",
                    (long long)S, k, need, comet::kStaticSelectScratchBytes);
    e = comet::static_select_scratch(&a.scratch);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(select scratch)");
    e = comet::launch_select(dtype, a, (cudaStream_t)stream);
    return e == cudaSuccess ? COMET_OK : cuda_fail(e, "select launch");
}

comet_status comet_scan_classify(comet_ctx *ctx, comet_dtype dtype, const comet_field *field,
                                 const comet_scan_params *params, const void *points,
                                 const int32_t *n_valid, const int8_t *charge, int64_t S,
                                 const int64_t *seed_index, const void *wires, int32_t W,
                                 int32_t ldw, const int32_t *hit_offsets, const void *drift,
                                 uint8_t *hit_mask, uint8_t *hit_class, void *dca_wire,
                                 int32_t update_mask, comet_stream stream)
{
    if (!ctx) return fail(COMET_ERR_INVALID_ARG, "ctx is NULL");
    CHECK(check_dtype(dtype));
    CHECK(check_field(field));
    CHECK(check_params(params, true));
    if (S < 1) return fail(COMET_ERR_INVALID_ARG, "S must be >= 1");
    CHECK(check_hits(dtype, wires, W, ldw, hit_offsets, drift, hit_mask));
    if (W == 0) return COMET_OK;
    if (!points || !n_valid || !charge || !seed_index || !hit_class)
        return fail(COMET_ERR_INVALID_ARG, "points, n_valid, charge, seed_index and hit_class are required");
    if (!aligned(points, esize(dtype)) || !aligned(n_valid, 4) || !aligned(seed_index, 8) ||
        (dca_wire && !aligned(dca_wire, esize(dtype))))
        return fail(COMET_ERR_INVALID_ARG, "an array is misaligned for its element type");
    DeviceGuard g(ctx->device);
    if (g.err != cudaSuccess) return cuda_fail(g.err, "cudaSetDevice");
    comet::ClsArgs a;
    fill_cls(ctx, dtype, params, points, n_valid, charge, S, seed_index, wires, W, ldw, hit_offsets, drift,
             hit_mask, hit_class, dca_wire, update_mask, &a);
    cudaError_t e = comet::launch_classify(dtype, *field, a, (cudaStream_t)stream);
    return e == cudaSuccess ? COMET_OK : cuda_fail(e, "classify launch");
}

} // extern "C"
