// Host-side pieces shared by the C ABI translation units (comet_scan.cu, batch.cu): the context
// object, argument validation, and the builders of the kernels' argument blocks.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "comet_scan.h"
#include "internal.h"

#define COMET_CHECK(expr)                                                                          \
    do {                                                                                           \
        comet_status _s = (expr);                                                                  \
        if (_s != COMET_OK) return _s;                                                             \
    } while (0)

namespace comet {
namespace detail {

// Pinned host and device staging of comet_scan_batch (sized by the caps of the last update).
struct BatchState {
    void *host = nullptr, *dev = nullptr;
    cudaEvent_t copied = nullptr;          // recorded after each descriptor copy
    bool recorded = false, ready = false;
    cudaStream_t last_stream = nullptr;
    comet_batch_caps caps{};
    int dtype = -1, stride = 0, B = 0;
    unsigned dca_ctas = 0;
    size_t host_bytes = 0;
    BatchLaunch launch{};
    void release();
};

comet_status fail(comet_status st, const char *fmt, ...);
comet_status cuda_fail(cudaError_t e, const char *where);

// Makes a device current for the scope of a call and restores the caller's device afterwards.
struct DeviceGuard {
    int prev = -1;
    cudaError_t err = cudaSuccess;
    explicit DeviceGuard(int dev);
    ~DeviceGuard();
};

size_t esize(comet_dtype dt);
bool aligned(const void *p, size_t a);
bool bounds_aligned(const void *b);
comet_status check_dtype(comet_dtype dt);
comet_status check_field(const comet_field *f);
comet_status check_params(const comet_scan_params *p, bool need_hits);
comet_status check_hits(comet_dtype dt, const void *wires, int32_t W, int32_t ldw, const int32_t *offs,
                        const void *drift, const void *mask);
int n_rec_of(const comet_scan_params *p);

// Segmentation and reaches of the closest-state search (identical for propagate and dca).
struct SearchGeometry {
    int G0, G1;
    double R0, R1, half_rec, h_rec;
};
SearchGeometry search_geometry(comet_dtype dtype, const comet_scan_params *p);

// Argument blocks of the kernels, from validated arguments.
void fill_lat(const comet_lattice &lat, int8_t *charge_out, LatArgs *a);
void fill_lat_table(const LatArgs &a, LatTable *t);
void fill_prop(comet_dtype dtype, const comet_scan_params *p, const SearchGeometry &sg, const void *seeds,
               const int8_t *charge, int64_t S, void *points, int32_t *n_valid, void *bounds, PropArgs *a);
void fill_dca(comet_ctx *ctx, comet_dtype dtype, const comet_scan_params *p, const SearchGeometry &sg,
              const void *points, const int32_t *n_valid, const int8_t *charge, int64_t S,
              const void *bounds, const void *wires, int32_t W, int32_t ldw, const int32_t *offs,
              const void *drift, const uint8_t *mask, void *rss, int32_t *n_in, void *dca_out,
              int32_t *n_unconverged, DcaArgs *a);
void fill_cls(comet_ctx *ctx, comet_dtype dtype, const comet_scan_params *p, const void *points,
              const int32_t *n_valid, const int8_t *charge, int64_t S, const int64_t *seed_index,
              const void *wires, int32_t W, int32_t ldw, const int32_t *offs, const void *drift,
              uint8_t *mask, uint8_t *hit_class, void *dca_wire, int32_t update_mask, ClsArgs *a);

} // namespace detail
} // namespace comet

struct comet_ctx {
    int device;
    void *scratch = nullptr;     // comet_scan_select's per-block partial results
    size_t scratch_bytes = 0;
    int32_t *status = nullptr;   // device status word (bit 0: bulk-copy timeout, bit 1: bad seed index)
    uint64_t copy_wait_ns = 2000000000ull;   // limit of a kernel's wait for a staging bulk copy
    int dca_ctas_per_sm = 0;                 // cap of the persistent DCA launch (0: as many as fit)
    int dca_chunk_wires = 0;                 // wires per chunk of the DCA's sums (0: automatic)
    int record_blocks = 1;                   // FP64 axial recording of few seeds by super-segment
    void *dca_part = nullptr;    // comet_scan_dca's per-chunk partial sums
    size_t dca_part_bytes = 0;
    uint32_t *dca_arrive = nullptr;   // per-group arrival counters (kept zero between launches)
    void *dca_best = nullptr;         // per-CTA slots of comet_scan_dca's fused selection
    int64_t dca_best_cap = 0;         // slots
    size_t dca_arrive_n = 0;
    comet::detail::BatchState batch;
};
