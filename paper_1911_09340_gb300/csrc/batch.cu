// Batches of events in single launches: the host side of comet_scan_batch / comet_scan_batch_update.
//
// A batch is one turn partition of up to caps.max_events events.  comet_scan_batch_update packs, in
// the context's pinned staging buffer, one BatchEvent per event (the same argument blocks the
// single-event calls build), the per-event prefix arrays that map each block of a batched launch to
// its event, and the CTA -> event map of the persistent DCA launch (CTAs apportioned to the events
// by their number of 32-seed groups, at least one each).  comet_scan_batch then enqueues one copy
// of that buffer to the device and the batched launches lattice -> propagate -> dca -> select ->
// classify.  Every grid size and device offset follows the caps alone, so the enqueued work can be
// captured in a CUDA graph once and replayed for any other batch within the same caps after a new
// comet_scan_batch_update.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "comet_scan.h"
#include "internal.h"
#include "scan_ctx.h"

namespace {

using comet::BatchEvent;
using comet::BatchLaunch;

size_t round_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

struct Layout {
    int E;                   // event slots = caps.max_events
    int64_t nb_sel;          // select pass-1 blocks per event at most
    unsigned lat_blocks, prop_blocks, sel_blocks, cls_blocks, dca_ctas;
    size_t ev, lat, prop, sel, cls, map, host_bytes, counters, part, scratch, dev_bytes;
    size_t scratch_per_event;
};

Layout make_layout(const comet_batch_caps &c, comet_dtype dt, unsigned dca_ctas)
{
    Layout L;
    L.E = c.max_events;
    const int64_t chunk = comet::select_chunk();
    L.nb_sel = (c.max_seeds + chunk - 1) / chunk;
    L.lat_blocks = (unsigned)((c.max_total_seeds + 255) / 256 + L.E);
    L.prop_blocks = (unsigned)((c.max_total_seeds + 127) / 128 + L.E);
    L.sel_blocks = (unsigned)((c.max_total_seeds + chunk - 1) / chunk + L.E);
    L.cls_blocks = (unsigned)(((int64_t)c.max_total_wires + 7) / 8 + L.E);
    L.dca_ctas = dca_ctas;
    size_t o = 0;
    L.ev = o;
    o = round_up(o + sizeof(BatchEvent) * L.E, 256);
    L.lat = o;
    o = round_up(o + sizeof(int64_t) * (L.E + 1), 256);
    L.prop = o;
    o = round_up(o + sizeof(int64_t) * (L.E + 1), 256);
    L.sel = o;
    o = round_up(o + sizeof(int64_t) * (L.E + 1), 256);
    L.cls = o;
    o = round_up(o + sizeof(int64_t) * (L.E + 1), 256);
    L.map = o;                               // DCA chunk prefix
    o = round_up(o + sizeof(int64_t) * (L.E + 1), 256);
    L.host_bytes = o;                        // copied host -> device on every batch
    L.counters = o;                          // the DCA item counter
    o = round_up(o + sizeof(unsigned long long), 256);
    L.part = o;                              // the DCA CTAs' partial sums
    o = round_up(o + (size_t)dca_ctas * comet::kDcaBatchSub * 32 * (2 * (dt == COMET_F32 ? 4 : 8) + 4), 256);
    L.scratch_per_event = round_up((size_t)L.nb_sel * (sizeof(int64_t) + (dt == COMET_F32 ? 4 : 8)), 256);
    L.scratch = o;
    o += L.scratch_per_event * L.E;
    L.dev_bytes = o;
    return L;
}

bool same_caps(const comet_batch_caps &a, const comet_batch_caps &b)
{
    return a.max_events == b.max_events && a.max_seeds == b.max_seeds &&
           a.max_total_seeds == b.max_total_seeds && a.max_wires == b.max_wires &&
           a.max_total_wires == b.max_total_wires && a.dca_ctas_per_sm == b.dca_ctas_per_sm &&
           a.dca_item_groups == b.dca_item_groups;
}

} // namespace

using comet::detail::fail;
using comet::detail::cuda_fail;

extern "C" {

comet_status comet_scan_batch_update(comet_ctx *ctx, comet_dtype dtype, const comet_field *field,
                                     const comet_scan_params *params, const comet_batch_caps *caps,
                                     const comet_batch_event *events, int32_t B)
{
    using namespace comet::detail;
    if (!ctx) return fail(COMET_ERR_INVALID_ARG, "ctx is NULL");
    COMET_CHECK(check_dtype(dtype));
    COMET_CHECK(check_field(field));
    COMET_CHECK(check_params(params, true));
    if (!caps) return fail(COMET_ERR_INVALID_ARG, "caps is NULL");
    if (caps->max_events < 1 || caps->max_events > 65536 || caps->max_seeds < 1 ||
        caps->max_total_seeds < caps->max_seeds || caps->max_wires < 0 || caps->max_wires > 1024 ||
        caps->max_total_wires < caps->max_wires)
        return fail(COMET_ERR_INVALID_ARG, "caps out of range (max_wires <= 1024; totals >= per-event maxima)");
    if (B < 0 || B > caps->max_events) return fail(COMET_ERR_INVALID_ARG, "B must be in 0 .. caps.max_events");
    if (B > 0 && !events) return fail(COMET_ERR_INVALID_ARG, "events is NULL");
    DeviceGuard g(ctx->device);
    if (g.err != cudaSuccess) return cuda_fail(g.err, "cudaSetDevice");

    int per_sm = comet::dca_persistent_ctas_per_sm(dtype, *field, caps->max_wires);
    if (per_sm < 1) return fail(COMET_ERR_CUDA, "no resident DCA CTA for %d wires", caps->max_wires);
    if (caps->dca_ctas_per_sm < 0) return fail(COMET_ERR_INVALID_ARG, "caps.dca_ctas_per_sm must be >= 0");
    if (caps->dca_item_groups < 0 || caps->dca_item_groups > comet::kDcaBatchSub)
        return fail(COMET_ERR_INVALID_ARG, "caps.dca_item_groups must be in 0 .. %d", comet::kDcaBatchSub);
    if (caps->dca_ctas_per_sm > 0 && caps->dca_ctas_per_sm < per_sm) per_sm = caps->dca_ctas_per_sm;
    const unsigned dca_ctas = (unsigned)(per_sm * comet::device_sm_count());
    const Layout L = make_layout(*caps, dtype, dca_ctas);

    // (re)allocate the staging buffers when the caps or the dtype change
    BatchState &bs = ctx->batch;
    if (!bs.host || !same_caps(bs.caps, *caps) || bs.dtype != (int)dtype || bs.dca_ctas != dca_ctas) {
        cudaError_t e = cudaDeviceSynchronize();
        if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceSynchronize");
        bs.release();
        e = cudaMallocHost(&bs.host, L.host_bytes);
        if (e == cudaSuccess) e = cudaMalloc(&bs.dev, L.dev_bytes);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&bs.copied, cudaEventDisableTiming);
        if (e != cudaSuccess) {
            bs.release();
            return e == cudaErrorMemoryAllocation ? fail(COMET_ERR_NO_MEMORY, "batch staging (%zu B)", L.dev_bytes)
                                                  : cuda_fail(e, "batch staging");
        }
        bs.caps = *caps;
        bs.dtype = (int)dtype;
        bs.dca_ctas = dca_ctas;
    } else if (bs.recorded) {
        // the previous batch's copy of this buffer must have left before it is rewritten
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        cudaStreamIsCapturing(bs.last_stream, &cs);
        if (cs == cudaStreamCaptureStatusNone) {
            cudaError_t e = cudaEventSynchronize(bs.copied);
            if (e != cudaSuccess) return cuda_fail(e, "cudaEventSynchronize");
        }
    }

    unsigned char *H = (unsigned char *)bs.host;
    unsigned char *D = (unsigned char *)bs.dev;
    BatchEvent *ev = (BatchEvent *)(H + L.ev);
    int64_t *lat = (int64_t *)(H + L.lat), *prop = (int64_t *)(H + L.prop);
    int64_t *sel = (int64_t *)(H + L.sel), *cls = (int64_t *)(H + L.cls);
    int64_t *dstart = (int64_t *)(H + L.map);
    std::memset(H, 0, L.host_bytes);

    const size_t es = esize(dtype);
    int64_t tot_seeds = 0, tot_wires = 0;
    std::vector<int64_t> groups(L.E, 0);
    lat[0] = prop[0] = sel[0] = cls[0] = dstart[0] = 0;
    for (int e = 0; e < L.E; ++e) {
        BatchEvent &be = ev[e];
        const comet_batch_event *x = e < B ? &events[e] : nullptr;
        int64_t S = 0;
        int W = 0;
        if (x && x->active) {
            int64_t prod = 1;
            for (int d = 0; d < 4; ++d) {
                if (x->lattice.counts[d] < 1) return fail(COMET_ERR_INVALID_ARG, "event %d: lattice counts must be >= 1", e);
                prod *= x->lattice.counts[d];
                if (!std::isfinite(x->lattice.centre[d]) || !std::isfinite(x->lattice.half_width[d]))
                    return fail(COMET_ERR_INVALID_ARG, "event %d: lattice centre/half_width must be finite", e);
            }
            S = prod;
            W = x->W;
            if (S > caps->max_seeds) return fail(COMET_ERR_INVALID_ARG, "event %d: %lld seeds > caps.max_seeds", e, (long long)S);
            if (W < 0 || W > caps->max_wires) return fail(COMET_ERR_INVALID_ARG, "event %d: W out of 0 .. caps.max_wires", e);
            if (x->n_steps < 1) return fail(COMET_ERR_INVALID_ARG, "event %d: n_steps must be >= 1", e);
            if (x->lattice.charge < -128 || x->lattice.charge > 127) return fail(COMET_ERR_INVALID_ARG, "event %d: charge must fit int8", e);
            COMET_CHECK(check_hits(dtype, x->wires, W, x->ldw, x->hit_offsets, x->drift, x->hit_mask));
            const void *need[] = {x->seeds, x->charge, x->points, x->n_valid, x->bounds, x->rss, x->n_in,
                                  x->best_idx};
            for (const void *q : need)
                if (!q) return fail(COMET_ERR_INVALID_ARG, "event %d: a required array is NULL", e);
            if (!aligned(x->seeds, es) || !aligned(x->points, es) || !aligned(x->rss, es) ||
                !aligned(x->n_valid, 4) || !aligned(x->n_in, 4) || !aligned(x->best_idx, 8) ||
                !bounds_aligned(x->bounds) || (x->best_rss && !aligned(x->best_rss, es)))
                return fail(COMET_ERR_INVALID_ARG, "event %d: an array is misaligned", e);
            if (W > 0 && !x->hit_class) return fail(COMET_ERR_INVALID_ARG, "event %d: hit_class is required", e);
            tot_seeds += S;
            tot_wires += W;
        }
        be.S = S;
        lat[e + 1] = lat[e] + (S + 255) / 256;
        prop[e + 1] = prop[e] + (S + 127) / 128;
        sel[e + 1] = sel[e] + (S + comet::select_chunk() - 1) / comet::select_chunk();
        cls[e + 1] = cls[e] + (W > 0 && S > 0 ? (W + 7) / 8 : 0);
        groups[e] = (S + 31) / 32;
        const int nc_e = comet::dca_wire_chunks(W, S, ctx->dca_chunk_wires);
        int gpi = comet::dca_batch_groups(nc_e);
        if (caps->dca_item_groups > 0 && caps->dca_item_groups < gpi) gpi = caps->dca_item_groups;
        dstart[e + 1] = dstart[e] + (groups[e] + gpi - 1) / gpi;
        if (!S) continue;

        comet_scan_params p = *params;
        p.n_steps = x->n_steps;
        const SearchGeometry sg = search_geometry(dtype, &p);
        // lattice
        fill_lat(x->lattice, x->charge, &be.lat);
        fill_lat_table(be.lat, &be.lat_tab);
        be.seeds = x->seeds;
        // propagate
        fill_prop(dtype, &p, sg, x->seeds, x->charge, S, x->points, x->n_valid, x->bounds, &be.prop);
        // dca (the counter is set per CTA on the device)
        fill_dca(ctx, dtype, &p, sg, x->points, x->n_valid, x->charge, S, x->bounds, x->wires, W, x->ldw,
                 x->hit_offsets, x->drift, x->hit_mask, x->rss, x->n_in, nullptr, x->n_unconverged, &be.dca);
        be.dca.batch_groups = gpi;
        // select (k = 1)
        be.sel.rss = x->rss;
        be.sel.S = S;
        be.sel.k = 1;
        be.sel.idx_out = x->best_idx;
        be.sel.rss_out = x->best_rss;
        be.sel.scratch = D + L.scratch + L.scratch_per_event * e;
        be.sel.n_blocks = (int)((S + comet::select_chunk() - 1) / comet::select_chunk());
        // classify (update the mask)
        if (W > 0)
            fill_cls(ctx, dtype, &p, x->points, x->n_valid, x->charge, S, x->best_idx, x->wires, W, x->ldw,
                     x->hit_offsets, x->drift, x->hit_mask, x->hit_class, nullptr, 1, &be.cls);
    }
    if (tot_seeds > caps->max_total_seeds) return fail(COMET_ERR_INVALID_ARG, "batch has %lld seeds > caps.max_total_seeds", (long long)tot_seeds);
    if (tot_wires > caps->max_total_wires) return fail(COMET_ERR_INVALID_ARG, "batch has %lld wires > caps.max_total_wires", (long long)tot_wires);

    bs.B = L.E;
    bs.launch.ev = (const BatchEvent *)(D + L.ev);
    bs.launch.lat_start = (const int64_t *)(D + L.lat);
    bs.launch.prop_start = (const int64_t *)(D + L.prop);
    bs.launch.sel_start = (const int64_t *)(D + L.sel);
    bs.launch.cls_start = (const int64_t *)(D + L.cls);
    bs.launch.dca_start = (const int64_t *)(D + L.map);
    bs.launch.chunk_counter = (unsigned long long *)(D + L.counters);
    bs.launch.dca_part = D + L.part;
    bs.launch.B = L.E;
    bs.launch.lat_blocks = L.lat_blocks;
    bs.launch.prop_blocks = L.prop_blocks;
    bs.launch.sel_blocks = L.sel_blocks;
    bs.launch.cls_blocks = L.cls_blocks;
    bs.launch.dca_ctas = L.dca_ctas;
    bs.launch.W_max = caps->max_wires;
    bs.host_bytes = L.host_bytes;
    bs.stride = params->stride;
    bs.ready = true;
    return COMET_OK;
}

comet_status comet_scan_batch(comet_ctx *ctx, comet_dtype dtype, const comet_field *field,
                              const comet_scan_params *params, const comet_batch_caps *caps,
                              const comet_batch_event *events, int32_t B, comet_stream stream)
{
    using namespace comet::detail;
    if (events || B > 0) COMET_CHECK(comet_scan_batch_update(ctx, dtype, field, params, caps, events, B));
    if (!ctx) return fail(COMET_ERR_INVALID_ARG, "ctx is NULL");
    BatchState &bs = ctx->batch;
    if (!bs.ready) return fail(COMET_ERR_INVALID_ARG, "no batch prepared (call comet_scan_batch_update)");
    if (bs.dtype != (int)dtype || bs.stride != params->stride)
        return fail(COMET_ERR_INVALID_ARG, "dtype / stride differ from the prepared batch");
    DeviceGuard g(ctx->device);
    if (g.err != cudaSuccess) return cuda_fail(g.err, "cudaSetDevice");
    cudaStream_t st = (cudaStream_t)stream;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaError_t e = cudaStreamIsCapturing(st, &cs);
    if (e == cudaSuccess) e = cudaMemcpyAsync(bs.dev, bs.host, bs.host_bytes, cudaMemcpyHostToDevice, st);
    // under capture the record becomes a node of the graph, so that a replay records it too
    if (e == cudaSuccess)
        e = cs == cudaStreamCaptureStatusActive ? cudaEventRecordWithFlags(bs.copied, st, cudaEventRecordExternal)
                                                : cudaEventRecord(bs.copied, st);
    if (e != cudaSuccess) return cuda_fail(e, "batch descriptor copy");
    bs.recorded = true;
    bs.last_stream = st;
    const BatchLaunch &L = bs.launch;
    if ((e = comet::launch_lattice_batch(dtype, L, st)) != cudaSuccess) return cuda_fail(e, "batch lattice");
    if ((e = comet::launch_propagate_batch(dtype, *field, bs.stride, L, st)) != cudaSuccess)
        return cuda_fail(e, "batch propagate");
    if ((e = comet::launch_dca_batch(dtype, *field, L, st)) != cudaSuccess) return cuda_fail(e, "batch dca");
    if ((e = comet::launch_select_batch(dtype, L, st)) != cudaSuccess) return cuda_fail(e, "batch select");
    if ((e = comet::launch_classify_batch(dtype, *field, L, st)) != cudaSuccess) return cuda_fail(e, "batch classify");
    return COMET_OK;
}

} // extern "C"
