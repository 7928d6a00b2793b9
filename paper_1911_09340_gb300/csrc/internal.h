// Launchers shared between the C-ABI layer (comet_scan.cu) and the kernel translation units.
// Arguments arrive here already validated.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "comet_scan.h"

namespace comet {

// A float-float value hi + lo (device.cuh holds its arithmetic).
struct ff {
    float hi, lo;
};

struct LatArgs {
    double vx, vy;
    double centre[4], half_width[4];
    int counts[4];
    int charge;
    int8_t *charge_out;
};

// Node values of a lattice's four dimensions and cos / sin of its phi nodes, computed once on the
// host (per block on the device they cost double divisions and sincos in every block); use = 0
// when the counts exceed the table (the kernel then tabulates per block).
constexpr int kLatParamNodes = 128;
constexpr int kLatParamPhi = 64;
struct LatTable {
    int use;
    double node[kLatParamNodes];
    double cphi[kLatParamPhi], sphi[kLatParamPhi];
};

struct PropArgs {
    const void *seeds;
    const int8_t *charge;
    int64_t S;
    void *points;
    int32_t *n_valid;
    void *bounds;          // optional: segment bounding spheres per 32-seed group (float4)
    double h, zmin, zmax, rmax;
    int n_steps, stride, n_rec;
    int G0, G1;            // segment sizes of the closest-state search
    double R0, R1;         // segment reaches (m), margins included
    // FP32 copies rounded on the host: h as a float-float pair; zmin, zmax, rmax^2, R0, R1
    ff h_ff;
    float lim_f[5];
};

struct DcaArgs {
    const void *points;
    const void *bounds;    // optional: written by propagate with the same params
    const int32_t *n_valid;
    const int8_t *charge;
    int64_t S;
    int n_rec;
    const void *wires;
    int W, ldw;
    const int32_t *offs;
    const void *drift;
    const uint8_t *mask;
    void *rss;
    int32_t *n_in;
    void *dca_out;
    int32_t *n_unconv;
    int32_t *status;       // device status word of the context (bit 0: a bulk-copy wait timed out)
    int32_t *counter;      // device work counter (context-owned; zeroed before each launch)
    uint64_t wait_ns;      // limit of a wait for a staging bulk copy (0: give up at once)
    int max_ctas_per_sm;   // persistent launch: at most this many CTAs per SM (0: as many as fit)
    int batch_groups;      // batched launch: 32-seed groups per CTA item (0: kDcaBatchSub / n_chunks)
    // optional k = 1 selection inside the launch: the seed of lowest RSS and its RSS, through
    // per-CTA slots (int64 index [slots_cap], then T value [slots_cap]; slots_cap >= the grid) and
    // a CTA arrival counter kept at zero between launches
    int64_t *best_idx_out;
    void *best_rss_out;
    void *best_slots;
    int64_t best_slots_cap;
    uint32_t *best_counter;
    double lambda, tol;
    double R0;             // super-segment radius (m), margins included
    double R1;             // level-1 segment radius (m), margins included
    double half_rec;       // half a recording interval (m), margins included
    double h_rec;          // recording interval stride*h (m): reach of the local refinement
    // the four scalars above rounded to float on the host: the FP32 kernel reads these, so that
    // no double-to-float conversion is re-done inside its loops
    float lambda_f, tol_f, half_rec_f, h_rec_f;
    // rounding margin of the closest-state search (m; 4e-6 FP32, 1e-9 FP64) and its float copy
    double margin;
    float margin_f;
    int max_iter;
    int G0;                // recorded states per super-segment
    int G1;                // recorded states per level-1 segment
    int exact_all;         // refine every wire (dca_out requested)
    // The wires are cut into n_chunks chunks (dca_wire_chunks(W, S)); a seed's RSS is the sum of its
    // per-chunk compensated partial sums, added in chunk order.  With `part` and `arrive` given,
    // the persistent kernel schedules (group, chunk) items across warps: partial sums go to part
    // ([n_chunks][S] hi, [n_chunks][S] lo in T, then [n_chunks][S] int32 n_in) and the last warp
    // to finish a group (arrive[group] counts, reset to 0 afterwards) adds them up.  Without them a
    // warp does all chunks of its group itself, with the same arithmetic.
    int n_chunks;
    void *part;
    uint32_t *arrive;
};

// Wire chunks of the DCA's per-seed sums for W wires and S seeds (W <= 1024; 1 otherwise):
// ceil(W / 32), or more, narrower chunks (at least 4 wires each, at most kDcaBatchSub) when
// fewer than 4096 (32-seed group, chunk) items would result; chunk_wires > 0 (the context's
// setting) fixes the width instead (at most kDcaBatchSub chunks).  The same function serves the
// single-event and the batched launches, so both sum in the same order.
int dca_wire_chunks(int W, int64_t S, int chunk_wires);

struct SelArgs {
    const void *rss;
    int64_t S;
    int k;
    int64_t *idx_out;
    void *rss_out;
    void *scratch;         // per-block partial results
    int n_blocks;
};

struct ClsArgs {
    const void *points;
    const int32_t *n_valid;
    const int8_t *charge;
    int64_t S;
    int n_rec;
    const int64_t *seed_index;
    const void *wires;
    int W, ldw;
    const int32_t *offs;
    const void *drift;
    uint8_t *mask;
    uint8_t *hit_class;
    void *dca_wire;
    int32_t *status;       // bit 1: seed_index out of range
    double lambda, tol, h_rec;
    int max_iter;
    int update_mask;
};

// Levenberg-Marquardt step over S seeds (comet_scan_lm_step).
struct LmArgs {
    int64_t S;
    double *theta, *srss, *jtj, *jtr;
    double *theta_try;
    const double *srss_try, *jtj_try, *jtr_try;
    double *mu;
    double up, down, mu_min, mu_max;
    int first;
};
cudaError_t launch_lm_step(const LmArgs &a, cudaStream_t st);

// SM version (major * 10 + minor) of the library's device code, read from a kernel's attributes.
cudaError_t kernel_binary_version(int *version);

cudaError_t launch_lattice(comet_dtype dt, const LatArgs &a, const LatTable &t, void *seeds, int64_t S,
                           cudaStream_t st);
cudaError_t launch_lattice_refined(comet_dtype dt, const LatArgs &a, const double *refs,
                                   const int32_t *n_refs, int K, void *seeds, int64_t S,
                                   cudaStream_t st);

struct RefArgs {
    const void *seeds;
    int64_t S;
    const int64_t *idx;
    int M, K;
    double half_width[4];
    double *refs_out;
    int32_t *n_refs_out;
};
cudaError_t launch_refine_refs(comet_dtype dt, const RefArgs &a, cudaStream_t st);

struct JacArgs {
    const double *theta;   // [S][4] (z0, phi, pz, pT)
    int64_t S;
    double vx, vy, bz;
    int charge;
    double h, h_rec, zmin, zmax, rmax2, tol, lambda, tau;
    int stride, n_rec, max_iter;
    const void *wires;
    int W, ldw;
    const int32_t *offs;
    const double *drift;
    const uint8_t *mask;
    double *work;          // [S][W][11]
    double *srss_out, *grad_out, *jtj_out, *jtr_out;
    double *grad6_out;     // optional [S][6]: gradient in the Cartesian seed (x, y, z, px, py, pz)
    double *dca_out, *jac_out;
    int32_t *n_unconv;
};
cudaError_t launch_jacobian(const JacArgs &a, cudaStream_t st);

constexpr int kDcaWarpsPerCta = 4;   // warps of a persistent DCA CTA (128 threads)
// Batched DCA: a CTA takes one item of an event -- dca_batch_groups(n_chunks) consecutive 32-seed
// groups, i.e. at most kDcaBatchSub (group, wire chunk) sub-items, which its warps share out.
constexpr int kDcaBatchSub = 64;
__host__ __device__ inline int dca_batch_groups(int n_chunks)
{
    const int g = kDcaBatchSub / (n_chunks > 0 ? n_chunks : 1);
    return g > 0 ? g : 1;
}

// ---- batches of events (one turn partition each) in single launches ---------------------------
// Every batched launch has a fixed grid; block b finds its event e and its block index inside the
// event from a prefix array start[0..B] (start[e] <= b < start[e+1]); blocks past start[B] exit.
struct BatchEvent {
    LatArgs lat;
    LatTable lat_tab;
    void *seeds;
    int64_t S;
    PropArgs prop;
    DcaArgs dca;
    SelArgs sel;
    ClsArgs cls;
};

struct BatchLaunch {
    const BatchEvent *ev;            // device [B]
    const int64_t *lat_start;        // device [B + 1] prefix of lattice blocks (256 seeds)
    const int64_t *prop_start;       // device [B + 1] prefix of propagate blocks (128 seeds)
    const int64_t *sel_start;        // device [B + 1] prefix of select pass-1 blocks
    const int64_t *cls_start;        // device [B + 1] prefix of classify blocks (8 wires)
    const int64_t *dca_start;        // device [B + 1] prefix of DCA items (dca_batch_groups groups)
    unsigned long long *chunk_counter;  // device [1]: next DCA item
    void *dca_part;                  // device: per DCA CTA, kDcaBatchSub x 32 partial sums (hi, lo in T; n_in int32)
    int B;
    unsigned lat_blocks, prop_blocks, sel_blocks, cls_blocks, dca_ctas;
    int W_max;                       // largest W of the caps (shared-memory layout of the DCA CTAs)
};

// event of block b and its block index inside the event; false when b is past the batch
__device__ __forceinline__ bool batch_find(const int64_t *start, int B, int64_t b, int &e, int64_t &lb)
{
    if (b >= start[B]) return false;
    int lo = 0, hi = B - 1;   // largest e with start[e] <= b
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (start[mid] <= b)
            lo = mid;
        else
            hi = mid - 1;
    }
    e = lo;
    lb = b - start[lo];
    return true;
}

cudaError_t launch_lattice_batch(comet_dtype dt, const BatchLaunch &L, cudaStream_t st);
cudaError_t launch_propagate_batch(comet_dtype dt, const comet_field &f, int stride, const BatchLaunch &L,
                                   cudaStream_t st);
cudaError_t launch_dca_batch(comet_dtype dt, const comet_field &f, const BatchLaunch &L, cudaStream_t st);
cudaError_t launch_select_batch(comet_dtype dt, const BatchLaunch &L, cudaStream_t st);
cudaError_t launch_classify_batch(comet_dtype dt, const comet_field &f, const BatchLaunch &L,
                                  cudaStream_t st);
// CTAs per SM of the persistent DCA kernel for a shared-memory layout of W wires
int dca_persistent_ctas_per_sm(comet_dtype dt, const comet_field &f, int W);
int device_sm_count();
int select_chunk();   // RSS entries per select pass-1 block


cudaError_t launch_gn_step(double *theta, int64_t S, const double *jtj, const double *jtr, double mu,
                           cudaStream_t st);
cudaError_t launch_propagate(comet_dtype dt, const comet_field &f, const PropArgs &a, bool blocks,
                             cudaStream_t st);
cudaError_t launch_dca(comet_dtype dt, const comet_field &f, const DcaArgs &a, cudaStream_t st);
void dca_segments(int n_rec, int *G0, int *G1);   // segment sizes of the closest-state search
cudaError_t launch_select(comet_dtype dt, const SelArgs &a, cudaStream_t st);
size_t select_scratch_bytes(comet_dtype dt, int64_t S, int k, int *n_blocks);
// Allocation-free selection: size of the file-scope scratch array and its device address on the
// current device (looked up on the first call per device).
constexpr size_t kStaticSelectScratchBytes = (size_t)1 << 20;
cudaError_t static_select_scratch(void **ptr);
cudaError_t launch_classify(comet_dtype dt, const comet_field &f, const ClsArgs &a, cudaStream_t st);

// Field kinds the kernels are specialised for.
enum class FieldKind { Axial, Uniform, Table };
inline FieldKind field_kind(const comet_field &f)
{
    if (f.kind == 1 || f.kind == 2) return FieldKind::Table;
    return (f.b[0] == 0.0 && f.b[1] == 0.0) ? FieldKind::Axial : FieldKind::Uniform;
}

} // namespace comet
