/*
 * comet_scan.h -- C ABI of the GB300 (sm_103a) brute-force seed scan for multi-turn electron
 * reconstruction in a cylindrical drift chamber (arXiv:1911.09340, Sec. 2).
 *
 * The scan of one turn partition is five calls on one CUDA stream, with no host synchronisation
 * between them:
 *
 *   comet_scan_lattice    seeds from the prior ranges of the seed components        (Sec. 2.1, 3.1)
 *   comet_scan_propagate  track recording: extrapolate every seed, record its states (Algorithm 1)
 *   comet_scan_dca        DCA of every (seed, wire) and the capped per-seed RSS      (Algorithm 2, Eq. 1)
 *   comet_scan_select     the seeds of lowest RSS                                     (Sec. 2.1)
 *   comet_scan_refine_refs, comet_scan_lattice_refined
 *                         sparse references and finer lattices around them            (Sec. 2.1)
 *   comet_scan_jacobian, comet_scan_gn_step
 *                         smoothed RSS, dD/dseed, Gauss-Newton steps for the best seeds
 *   comet_scan_batch, comet_scan_batch_update
 *                         one turn partition of many events in single launches
 *   comet_scan_classify   classify the selected seed's hits; mask them for the next   (Sec. 2.1, 3.1)
 *                         turn partition
 *
 * Conventions shared by every call
 *   - Units: metres, MeV/c, tesla.  Equations of motion in arc length s, with P0 = |p| of the seed
 *     and KAPPA = 299.792458 MeV/c per (T m):  dx/ds = p / P0,  dp/ds = (KAPPA q / P0) p x B(x).
 *   - Every array pointer is a DEVICE pointer owned by the caller (for example a torch tensor), unless
 *     stated otherwise; the library never frees it.  Element type "T" is float for COMET_F32 and
 *     double for COMET_F64.  Arrays are dense and C-ordered; "SoA [6][S]" means component-major
 *     (row c holds component c of every seed), the seed index running fastest.
 *   - Every call is asynchronous on `stream` (a cudaStream_t; NULL is the legacy default stream) and
 *     returns once its kernels are enqueued.  Arguments are validated on the host before anything is
 *     launched; an invalid argument returns COMET_ERR_INVALID_ARG and launches nothing.  A failed
 *     launch returns COMET_ERR_CUDA.  No call aborts, throws or prints.  comet_last_error() returns
 *     a message for the last non-OK status of the calling thread.
 *   - The library allocates device memory only inside a comet_ctx (comet_scan_select_noalloc
 *     aside): a status word at creation; lazily, on first need and grown when a larger call needs
 *     more, comet_scan_select's per-block partial results, comet_scan_dca's per-chunk partial sums
 *     and per-group arrival counters, and its selection slots (16 B per CTA, when best_idx_out is
 *     given); the batch staging buffers; all kept until comet_ctx_destroy.  A call that grows
 *     scratch calls cudaMalloc (comet_scan_select also synchronises the device first); make the
 *     largest such call once before capturing a stream.
 */
#ifndef COMET_SCAN_H
#define COMET_SCAN_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *comet_stream; /* a cudaStream_t */
typedef struct comet_ctx comet_ctx;

typedef enum {
    COMET_OK = 0,
    COMET_ERR_INVALID_ARG = 1,
    COMET_ERR_CUDA = 2,
    COMET_ERR_NO_MEMORY = 3,
    COMET_ERR_UNSUPPORTED = 5
} comet_status;

typedef enum { COMET_F32 = 0, COMET_F64 = 1 } comet_dtype;

/* Magnetic field (Sec. 2.2.1: the field "in the grid format" is copied to the device).
 *   kind 0: uniform field b (tesla).
 *   kind 1: trilinear interpolation of a float32 DEVICE table [3][nz][ny][nx] (component, z, y, x)
 *           whose node (ix, iy, iz) sits at origin + spacing * (ix, iy, iz).  A coordinate outside
 *           the grid is clamped to its edge.  The same float32 table serves both dtypes.
 *   kind 2: the same interpolation of the same values laid out [nz][ny][nx][4] (bx, by, bz, unused)
 *           float32, 16-byte aligned: one 16-byte load per grid node instead of three scalar loads
 *           in three planes.  Results are identical to kind 1 with the same values. */
typedef struct {
    int32_t kind;
    double b[3];
    const void *table;
    int32_t nx, ny, nz;
    double origin[3];
    double spacing;
} comet_field;

/* Scan parameters.
 *   h         RK4 step (m), > 0.  The paper's extrapolator is an adaptive RKN (Sec. 2.1); here the
 *             step is fixed.
 *   n_steps   RK4 steps per turn partition, >= 1.
 *   stride    record every stride-th state, >= 1; state 0 (the seed) is always recorded, so
 *             n_rec = n_steps / stride + 1 states per seed.
 *   lambda    the cutoff of Eq. 1 (m), > 0.
 *   tol       virtual-plane distance below which the DCA refinement stops (m), > 0
 *             (Algorithm 2's TOLERANCE).
 *   max_iter  maximum refinement steps per (seed, wire), >= 0.
 *   zmin, zmax, rmax  target region: recording stops after the first recorded state with
 *             z < zmin, z > zmax or x^2 + y^2 > rmax^2 (Algorithm 1's loop condition). */
typedef struct {
    double h;
    int32_t n_steps;
    int32_t stride;
    double lambda;
    double tol;
    int32_t max_iter;
    double zmin, zmax, rmax;
} comet_scan_params;

/* Cartesian seed lattice (Sec. 2.1: seeds are combined from grids over the prior ranges of each
 * seed component).  Dimensions: vertex z0, transverse-momentum azimuth phi, p_z, p_T.  Node i of a
 * dimension with n nodes sits at centre + half_width * (2i/(n-1) - 1) (the centre alone when
 * n = 1).  Seed = (vx, vy, z0, pT cos phi, pT sin phi, pz), of charge `charge` (units of e; -1 for
 * the electron, +1 for the positron of the paper's Sec. 5.1 outlook).
 * Seed numbering: the lattice is cut into blocks of b = (2, 4, 4, 1) nodes along (z0, phi, pz, pT)
 * (b = 1 along a dimension whose count is odd; b = 2 along phi or pz when its count is even but not
 * a multiple of 4).  Blocks are numbered row-major with z0 slowest, nodes inside a block row-major,
 * and seed s = block * (b0 b1 b2 b3) + node-in-block: consecutive seeds are lattice neighbours, and
 * pT (the parameter that separates tracks fastest along a turn) is not mixed inside a block. */
typedef struct {
    double vx, vy;
    double centre[4];
    double half_width[4];
    int32_t counts[4];
    int32_t charge;
} comet_lattice;

/* ---- context ----------------------------------------------------------------------------------
 * comet_ctx_create: binds a context to CUDA device `device` (>= 0) and returns it in *out.  It
 * allocates one 256-byte device status word (zeroed).  comet_ctx_destroy synchronises the device,
 * frees the context's device memory and the context; NULL is a no-op.  A context may be used from
 * one host thread at a time.
 * comet_ctx_status: synchronises the device and copies the status word to *flags (host pointer):
 *   bit 0  a kernel's wait for a shared-memory bulk copy exceeded its time limit (2 s unless
 *          comet_ctx_set_copy_wait changed it); the kernel then re-read the data with plain loads,
 *          so its results are still valid;
 *   bit 1  comet_scan_classify was given a seed index outside [0, S); its hit_class was zeroed.
 * comet_ctx_set_copy_wait: the longest (ns >= 0, in nanoseconds) that a kernel launched with this
 *   context waits for a shared-memory bulk copy before it gives up, re-reads the data with plain
 *   loads and sets status bit 0 (default 2e9).  0 makes every such wait give up at once, so that the
 *   plain-load path runs on every launch: a way to test it.  A copy that was given up on is still
 *   waited for (up to 2 s) before the kernel reuses or releases the shared memory it writes.
 *   Host-side setting; takes effect for calls enqueued after it.
 * comet_ctx_set_dca_ctas_per_sm: at most n (1 .. 64; 0 = as many as fit, the default) resident CTAs
 *   per SM for comet_scan_dca's persistent launch with this context: leaves room on every SM for
 *   kernels of other streams (for example the next turn partition's track recording) to run beside
 *   it.  Results do not depend on it.  Host-side setting; takes effect for calls enqueued after it.
 * comet_ctx_set_dca_chunk_wires: wires per chunk of comet_scan_dca's per-seed sums (and of the
 *   batched launch) with this context: 0 (the default) takes chunks of at most 32 wires, narrower
 *   when a call has few seeds; 4 .. 1024 fixes the width (at most 64 chunks).  The chunking is a
 *   work split and a summation order (the sum within each chunk, then over chunks), so FP32 RSS
 *   values change in their last bits with it; the batched and single-event launches of one
 *   context use the same chunks.
 * comet_ctx_set_record_blocks: 1 (the default) lets comet_scan_propagate record FP64 tracks in a
 *   uniform axial field with fewer than four 32-seed groups per SM one super-segment per warp, each
 *   started from the composed interval map of Algorithm 1's fixed RK4 step (the track recording
 *   otherwise runs one warp per 32 seeds from the first state to the last, and a few seeds leave
 *   most of the part idle); 0 always takes the one-warp-per-32-seeds recording.  The states agree
 *   to rounding (about 1e-13 m over 2,000 steps), not bit for bit; comet_scan_batch always records
 *   one warp per 32 seeds, so a context whose single-event results must equal its batched ones bit
 *   for bit sets 0.  Host-side setting; takes effect for calls enqueued after it.
 * comet_kernel_arch: writes to *sm_version (host pointer) the SM version the library's device code
 *   was compiled for, as major * 10 + minor (103 for sm_103a), read from a kernel's attributes on
 *   the current device.
 * comet_last_error: message of the calling thread's last non-OK status (static storage). */
comet_status comet_ctx_create(int device, comet_ctx **out);
void comet_ctx_destroy(comet_ctx *ctx);
comet_status comet_ctx_status(comet_ctx *ctx, int32_t *flags);
comet_status comet_ctx_set_copy_wait(comet_ctx *ctx, int64_t ns);
comet_status comet_ctx_set_dca_ctas_per_sm(comet_ctx *ctx, int32_t n);
comet_status comet_ctx_set_dca_chunk_wires(comet_ctx *ctx, int32_t wires);
comet_status comet_ctx_set_record_blocks(comet_ctx *ctx, int32_t on);
comet_status comet_kernel_arch(int32_t *sm_version);
const char *comet_last_error(void);

/* ---- a1: seed lattice -------------------------------------------------------------------------
 * Writes the S = counts[0]*counts[1]*counts[2]*counts[3] seeds of `lat` to seeds (SoA [6][S], T)
 * and, if charge_out is not NULL, lat->charge to charge_out ([S] int8).  Computed in double and
 * rounded to T.  S must equal the product of the counts and the charge must fit int8 (else
 * COMET_ERR_INVALID_ARG).  Paper: Sec. 2.1 (grid of seeds over prior ranges), Sec. 3.1. */
comet_status comet_scan_lattice(comet_ctx *ctx, comet_dtype dtype, const comet_lattice *lat,
                                void *seeds, int8_t *charge_out, int64_t S, comet_stream stream);

/* ---- a2/a3: track recording (Algorithm 1, Sec. 2.2.1) ------------------------------------------
 *   seeds    SoA [6][S] T: (x, y, z, px, py, pz) of each seed.
 *   charge   [S] int8: particle charge in units of e (the electron is -1); 0 gives a straight line.
 *   points   out, SoA [6][n_rec][S] T: recorded state k of seed s is points[c][k][s].  Entries past
 *            n_valid[s] are unspecified (left unwritten, or states extrapolated past the target
 *            region by the FP64 block recording below); no call reads them.
 *   n_valid  out, [S] int32: number of recorded states of each seed (1 .. n_rec).
 *   bounds   optional out (NULL to skip), [ceil(S/32)][200][4] float32, 16-byte aligned: search
 *            bounds for comet_scan_dca with the same params -- for each group of 32 consecutive
 *            seeds, the bounding spheres (x, y, z, radius) of its track segments (8 super-segments,
 *            24 level-1 segments each).  Writing them costs a few percent of this call and saves
 *            comet_scan_dca from rebuilding them.
 * One thread extrapolates one seed with fixed-step RK4.  The FP32 path carries each state component
 * as an unevaluated float pair (a compensated sum), so that 6,500 steps stay within a few um of FP64;
 * the recorded value is the leading float.  FP64 in a uniform axial field with fewer than four
 * 32-seed groups per SM records one super-segment per warp instead (comet_ctx_set_record_blocks);
 * it then also sets n_valid with a byte memset before its kernel. */
comet_status comet_scan_propagate(comet_ctx *ctx, comet_dtype dtype, const comet_field *field,
                                  const comet_scan_params *params, const void *seeds,
                                  const int8_t *charge, int64_t S, void *points, int32_t *n_valid,
                                  void *bounds, comet_stream stream);

/* ---- a4-a6: DCA finding and RSS (Algorithm 2, Eq. 1, Sec. 2.2.2) --------------------------------
 *   points, n_valid, charge, S   as written by comet_scan_propagate with the same params.
 *   bounds       optional (NULL: built here), the bounds comet_scan_propagate wrote for these
 *                points with the same params.
 *   wires        SoA [6][ldw] T: (a_x, a_y, a_z, u_x, u_y, u_z) of wire i in column i: a point on
 *                the wire and its unit direction.  ldw >= W is the row stride in elements.
 *   W            number of wires (>= 0).  W = 0 gives rss = 0 and n_in = 0.
 *   hit_offsets  [W+1] int32 CSR: the hits of wire i are hit_offsets[i] .. hit_offsets[i+1]-1;
 *                hit_offsets[0] = 0, non-decreasing.
 *   drift        [H] T: drift distance r of each hit (H = hit_offsets[W]).
 *   hit_mask     [H] uint8: non-zero marks a hit classified by an earlier turn partition; it is
 *                ignored here, and a wire whose hits are all masked leaves the sum.
 *   rss          out, [S] T: RSS = sum over wires with an unmasked hit of d_i^2, where
 *                d_i = min(min_j |D_i - r_ij|, lambda) and D_i is the DCA of the track to wire i
 *                (Eq. 1; the left and right hits of drift r sit at +-r across the wire, so
 *                min(d^L, d^R) = |D - r|).  Summed in ascending wire order within chunks of at
 *                most 32 wires (FP32 as a compensated TwoSum pair, FP64 plainly), the chunk sums
 *                then in chunk order: deterministic, independent of the GPU's scheduling.
 *   n_in         out, [S] int32: wires whose capped residual is below lambda.
 *   dca_out      optional out, [W][S] T (NULL to skip): D_i of every (wire, seed).  Requesting it
 *                computes the exact DCA of every wire; without it, a wire the track never comes
 *                within (max drift + lambda + half a recording interval; a whole interval at the
 *                first and the last recorded state, which the refinement can move beyond) of is
 *                known to contribute lambda^2 and is not refined.
 *   n_unconverged optional, device [1] int32 (NULL to skip): incremented by the number of
 *                (seed, wire) refinements that reached max_iter or met a track parallel to the wire.
 *                The caller zeroes it.  Non-convergence is reported only here, never through the
 *                return status: the count exists on the device once the kernel has run, and
 *                returning it would need a host synchronisation in every call.
 *   best_idx_out optional out, device [1] int64 (NULL to skip): the seed of lowest RSS, exactly
 *                as comet_scan_select with k = 1 gives it (ascending RSS, NaN after every number,
 *                ties by lowest seed index), selected inside this launch (Sec. 2.1: the best seed of
 *                the partition) -- no separate selection launches: each CTA folds its seeds into
 *                a slot, and the last CTA to finish (an arrival counter in the status word) folds
 *                the slots.  best_rss_out optional [1] T: its RSS (needs best_idx_out).
 * D_i: start from the recorded state closest to the wire line (ties: lowest index), then step along
 * the track by -d/|n| with one RK4 step, where n is the part of the unit direction perpendicular to
 * the wire and d the distance to the plane that contains the wire axis with normal n, until
 * |d| < tol (Algorithm 2's loop; the Newton step length is the reading of "the distance").
 * The closest recorded state is found exactly by a bounded search over the recorded states (recorded
 * states one recording interval apart are at most that arc length apart).  The kernel takes a
 * device work counter from the context: dca calls of one context must not overlap on the GPU.
 * With more than 32 wires the context also keeps per-chunk partial sums and per-group counters for
 * the kernel (grown on demand, at least twofold: a call that grows them allocates device memory). */
comet_status comet_scan_dca(comet_ctx *ctx, comet_dtype dtype, const comet_field *field,
                            const comet_scan_params *params, const void *points,
                            const int32_t *n_valid, const int8_t *charge, int64_t S,
                            const void *bounds, const void *wires, int32_t W, int32_t ldw, const int32_t *hit_offsets,
                            const void *drift, const uint8_t *hit_mask, void *rss, int32_t *n_in,
                            void *dca_out, int32_t *n_unconverged, int64_t *best_idx_out,
                            void *best_rss_out, comet_stream stream);

/* ---- a7: selection (Sec. 2.1; top-k for Sec. 3.1's "10 seeds at each side") ------------------
 *   rss      [S] T.
 *   k        1 .. 64, and k <= S.
 *   idx_out  out, [k] int64: the seeds of the k lowest RSS in ascending order; equal RSS ordered by
 *            seed index; NaN sorts after every number.
 *   rss_out  out, [k] T (may be NULL).
 * Uses the context's device scratch (allocated on first use). */
comet_status comet_scan_select(comet_ctx *ctx, comet_dtype dtype, const void *rss, int64_t S,
                               int32_t k, int64_t *idx_out, void *rss_out, comet_stream stream);

/* ---- iterative refinement: references for a finer scan (Sec. 2.1) --------------------------------
 * Sec. 2.1: the seeds of lowest RSS become reference points for the next scan, whose seeds are taken
 * in their vicinity with a finer granularity; the references are kept sparse enough that the new
 * seed sets do not overlap.
 *   seeds       SoA [6][S] T: the scanned seeds (as written by comet_scan_lattice or
 *               comet_scan_lattice_refined).
 *   idx         [M] int64 device: candidate seed indices in the order to consider them (ascending
 *               RSS, as comet_scan_select returns them); indices outside [0, S) are skipped.
 *   M           1 .. 1048576.
 *   half_width  HOST [4] double >= 0: half-widths (z0, phi, pz, pT) of the lattices that will be
 *               built around the references.
 *   K           1 .. 32: the most references to take.
 *   refs_out    out, [K][4] double device: lattice coordinates (z0, phi = atan2(py, px), pz,
 *               pT = hypot(px, py)) of each accepted reference, best first.
 *   n_refs_out  out, [1] int32 device: number accepted (1 .. K when any index is valid).
 * A candidate is accepted unless some accepted reference lies within 2 * half_width[d] of it in
 * every coordinate d (phi modulo 2 pi): the two new lattices would overlap.  One warp; the greedy
 * walk is sequential in the candidate order. */
comet_status comet_scan_refine_refs(comet_ctx *ctx, comet_dtype dtype, const void *seeds, int64_t S,
                                    const int64_t *idx, int32_t M, const double half_width[4],
                                    int32_t K, double *refs_out, int32_t *n_refs_out,
                                    comet_stream stream);

/* ---- iterative refinement: the finer lattices (Sec. 2.1) ------------------------------------------
 *   shape     lattice of comet_scan_lattice whose centre is ignored: vertex (vx, vy), half-widths,
 *             counts and charge of every new lattice.
 *   refs      [K][4] double device, n_refs [1] int32 device: as written by comet_scan_refine_refs.
 *   K         1 .. 32 lattices; seeds k*S1 .. (k+1)*S1 - 1 (S1 = product of shape.counts) form
 *             lattice k, centred at refs[k] while k < *n_refs and at refs[0] beyond (a repeat, so
 *             that the seed count stays K*S1 whatever the number of references).
 *   seeds     out, SoA [6][S] T with S = K * S1; charge_out out, [S] int8 (may be NULL).
 * Inside each lattice the seeds follow the blocked numbering of comet_scan_lattice. */
comet_status comet_scan_lattice_refined(comet_ctx *ctx, comet_dtype dtype, const comet_lattice *shape,
                                        const double *refs, const int32_t *n_refs, int32_t K,
                                        void *seeds, int8_t *charge_out, int64_t S,
                                        comet_stream stream);

/* ---- residual Jacobians and Gauss-Newton steps for the best seeds ---------------------------------
 * Refines a few seeds continuously instead of by a finer grid.  The paper scans grids because its
 * RSS (Eq. 1) is not smooth in the seed (Sec. 2.1); this call smooths the cap of Eq. 1 and gives the
 * derivatives needed for Gauss-Newton.
 *   Seeds are theta [S][4] double device = (z0, phi, pz, pT) with vertex (vx, vy) and `charge`, as
 *   in comet_scan_lattice.  dtype must be COMET_F64; the field must be uniform along z
 *   (kind 0 with b[0] = b[1] = 0), else COMET_ERR_UNSUPPORTED.  params as for the scan (h, n_steps,
 *   stride, target region, tol, max_iter, lambda).
 *   For each (seed, wire): D = the DCA exactly as comet_scan_dca finds it (closest recorded state,
 *   then the local virtual-plane refinement of Algorithm 2) and dD/dtheta by forward-mode
 *   derivatives of the recorded states (closed form in an axial field) and of the refinement steps
 *   at fixed lengths (at the point of closest approach the distance is stationary along the track).
 *   For each wire with an unmasked hit: e = min_j |D - r_j|, w = 1 / (1 + exp(-(lambda - e)/tau)),
 *   term = w e^2 + (1 - w) lambda^2 (Eq. 1 with a smooth cap; tau > 0, in metres).
 *   work       [S][W][11] double device scratch.
 *   srss_out   out, [S] double: sum of the terms in ascending wire order (the smoothed RSS).
 *   grad_out   out, [S][4] double: its gradient in theta.
 *   jtj_out    out, [S][4][4] double: sum over wires of w J J^T (J = dD/dtheta);
 *   jtr_out    out, [S][4] double: sum of w J (D - r_j*), the Gauss-Newton normal equations with
 *              the weights held fixed.
 *   dca_out    optional out, [S][W] double: D.   jac_out optional out, [S][W][4] double: dD/dtheta.
 *   grad6_out  optional out, [S][6] double: the gradient of the smoothed RSS in the Cartesian seed
 *              (x, y, z, px, py, pz) -- the vertex (x, y) enters the recorded positions additively.
 *   n_unconverged optional [1] int32 device, incremented for refinements that did not converge. */
comet_status comet_scan_jacobian(comet_ctx *ctx, comet_dtype dtype, const comet_field *field,
                                 const comet_scan_params *params, const double *theta, int64_t S,
                                 double vx, double vy, int32_t charge, const void *wires, int32_t W,
                                 int32_t ldw, const int32_t *hit_offsets, const void *drift,
                                 const uint8_t *hit_mask, double tau, double *work,
                                 double *srss_out, double *grad_out, double *jtj_out,
                                 double *jtr_out, double *dca_out, double *jac_out,
                                 double *grad6_out, int32_t *n_unconverged, comet_stream stream);

/* theta[s] += delta with (JTJ + mu diag(JTJ)) delta = -JTR (Cholesky; a seed whose matrix is not
 * positive definite keeps its theta).  theta [S][4], jtj [S][4][4], jtr [S][4]: double device, as
 * written by comet_scan_jacobian.  mu >= 0 (Levenberg-Marquardt damping). */
comet_status comet_scan_gn_step(comet_ctx *ctx, double *theta, int64_t S, const double *jtj,
                                const double *jtr, double mu, comet_stream stream);

/* Levenberg-Marquardt with a per-seed accept/reject of each trial, all on the device (double device
 * arrays, S in 1 .. 2^24):
 *   theta [S][4], srss [S], jtj [S][4][4], jtr [S][4]: the current (accepted) seeds and
 *       comet_scan_jacobian's outputs at them; replaced by the trial's where it is accepted;
 *   theta_try [S][4]: the trial seeds; overwritten with the next trial;
 *   srss_try, jtj_try, jtr_try: comet_scan_jacobian's outputs at theta_try (ignored, may be NULL,
 *       when first != 0);
 *   mu [S]: per-seed damping.
 * Unless first != 0, each seed's trial is accepted when its smoothed RSS is below the current one
 * (then mu *= down), else rejected (mu *= up); mu stays within [1e-12, 1e12].  Then the next trial
 * is theta_try = theta + delta with (JTJ + mu diag(JTJ)) delta = -JTR (delta = 0 when that matrix
 * is not positive definite).  up >= 1, 0 < down <= 1.  So the smoothed RSS of the current seeds
 * never increases: Gauss-Newton steps with the safeguard that the smoothed RSS (whose cap makes it
 * non-convex, Sec. 2.1) cannot climb. */
comet_status comet_scan_lm_step(comet_ctx *ctx, int64_t S, double *theta, double *srss, double *jtj,
                                double *jtr, double *theta_try, const double *srss_try,
                                const double *jtj_try, const double *jtr_try, double *mu, double up,
                                double down, int32_t first, comet_stream stream);

/* ---- batches of events in single launches (many events at once) ---------------------------------
 * One turn partition of up to caps.max_events events: for each active event its lattice, track
 * recording, DCA and RSS, selection (k = 1) and classification with the mask update, exactly as the
 * single-event calls with the same arguments compute them, but each step one launch for the whole
 * batch.  A launch's blocks are apportioned to the events by their sizes; the persistent DCA
 * launch's CTAs take chunks of 16 32-seed groups from one counter over all events, restaging an
 * event's wires when they move to it.  Shared by the batch: dtype, field and params except n_steps;
 * W <= 1024.
 *
 * comet_scan_batch_update (host work only) validates the events and packs their descriptors into
 * the context's pinned staging buffer; comet_scan_batch enqueues one copy of that buffer to the
 * device and the batched launches.  Grid sizes and device offsets follow the caps alone, so the
 * work comet_scan_batch enqueues can be captured once in a CUDA graph (stream capture) and replayed
 * for any batch with the same caps, dtype and stride after comet_scan_batch_update has packed it.
 * An update waits for the previous batch's descriptor copy to leave the staging buffer before it
 * rewrites it.  Calling comet_scan_batch with events packs them first (an update); with events =
 * NULL and B = 0 it enqueues the last packed batch.  The first update with new caps allocates the
 * staging buffers (and synchronises the device): make it before capturing.  An update whose caps or
 * dtype differ from the previous one frees and reallocates the staging buffers, so a graph captured
 * before it copies from freed memory: such a graph must not be replayed again (capture anew). */
typedef struct {
    int32_t max_events;        /* event slots per batch, 1 .. 65536 */
    int64_t max_seeds;         /* seeds of one event */
    int64_t max_total_seeds;   /* seeds of all events of a batch */
    int32_t max_wires;         /* wires of one event, <= 1024 */
    int32_t max_total_wires;   /* wires of all events of a batch */
    int32_t dca_ctas_per_sm;   /* resident CTAs per SM of the batched DCA launch; 0: as many as fit */
    int32_t dca_item_groups;   /* 32-seed groups per item of the batched DCA launch, 0 .. 64;
                                  0: 64 / (wire chunks of the event) */
} comet_batch_caps;

typedef struct {
    int32_t active;               /* 0: slot skipped, nothing read or written */
    comet_lattice lattice;        /* the event's turn partition; S = product of the counts */
    int32_t n_steps;              /* RK4 steps of this partition (params->n_steps is not used) */
    void *seeds;                  /* scratch, SoA [6][S] T */
    int8_t *charge;               /* scratch, [S] */
    void *points;                 /* scratch, SoA [6][n_rec][S] T, n_rec = n_steps/stride + 1 */
    int32_t *n_valid;             /* scratch, [S] */
    void *bounds;                 /* scratch, [ceil(S/32)][200][4] float32, 16-byte aligned */
    const void *wires;            /* SoA [6][ldw] T, as comet_scan_dca */
    int32_t W, ldw;
    const int32_t *hit_offsets;   /* [W+1] */
    const void *drift;            /* [H] T */
    uint8_t *hit_mask;            /* in/out [H]: the hits classified here are set to 1 */
    void *rss;                    /* out [S] T */
    int32_t *n_in;                /* out [S] */
    int64_t *best_idx;            /* out [1]: the seed of lowest RSS */
    void *best_rss;               /* out [1] T (may be NULL) */
    uint8_t *hit_class;           /* out [H] (required when W > 0) */
    int32_t *n_unconverged;       /* optional [1], incremented */
} comet_batch_event;

comet_status comet_scan_batch_update(comet_ctx *ctx, comet_dtype dtype, const comet_field *field,
                                     const comet_scan_params *params, const comet_batch_caps *caps,
                                     const comet_batch_event *events, int32_t B);
comet_status comet_scan_batch(comet_ctx *ctx, comet_dtype dtype, const comet_field *field,
                              const comet_scan_params *params, const comet_batch_caps *caps,
                              const comet_batch_event *events, int32_t B, comet_stream stream);

/* ---- selection without device allocation (the paper has no counterpart) -------------------------
 * Same result as comet_scan_select, for callers that cannot allocate device memory: for example a
 * process whose device memory is owned by a caching allocator or held to a fixed budget, where an
 * extra cudaMalloc can fail or fragment the pool, or a caller that cannot create a comet_ctx (whose
 * creation allocates).  It takes no context, allocates nothing and calls no cudaMalloc or cudaFree.
 *   Runs on the CURRENT device (cudaGetDevice); stream must belong to it.  Arguments as for
 *   comet_scan_select.
 *   Scratch: a 1 MiB file-scope device array, present on every device that loads the library until
 *   the process exits.  A call needs ceil(S / 2048) * k * (sizeof(T) + 8) + 64 bytes of it and is
 *   rejected with COMET_ERR_INVALID_ARG beyond 1 MiB (k = 1: S up to about 134 million FP64 or
 *   178 million FP32 seeds; k = 64: about 2.09 million FP64 or 2.79 million FP32).
 *   The arrays must be device memory of the current device (else COMET_ERR_INVALID_ARG).
 *   The first call on a device looks the array's device address up (cudaGetSymbolAddress, with that
 *   device current) and keeps it for the rest of the process; make that first call before any
 *   stream capture.  The kept address does not survive a reset of the device's primary context
 *   (cudaDeviceReset): do not call this function after such a reset in the same process.
 *   Every call shares the array and it keeps the last call's contents; nothing in it needs to start
 *   at zero (each call writes every entry it reads).  Calls that overlap on the GPU (other streams,
 *   other host threads) race on the array: serialise them. */
comet_status comet_scan_select_noalloc(comet_dtype dtype, const void *rss, int64_t S, int32_t k,
                                       int64_t *idx_out, void *rss_out, comet_stream stream);

/* ---- a8/a9: classification (Sec. 2.1) and the mask of the next turn partition (Sec. 3.1) -------
 *   points, n_valid, charge, S, wires, W, ldw, hit_offsets, drift  as for comet_scan_dca.
 *   seed_index  device [1] int64: the seed to classify (for example idx_out of comet_scan_select);
 *               read on the device, so no host synchronisation is needed.  Must be in [0, S).
 *   hit_mask    [H] uint8, read; when update_mask != 0 the classified hits are OR-ed into it.
 *   hit_class   out, [H] uint8: 1 for the closest unmasked hit of each wire whose |D - r| is below
 *               lambda (ties: lowest hit index), 0 otherwise.
 *   dca_wire    optional out, [W] T (NULL to skip): the selected seed's DCA to every wire.
 * The closest recorded state is found by exhaustive search here. */
comet_status comet_scan_classify(comet_ctx *ctx, comet_dtype dtype, const comet_field *field,
                                 const comet_scan_params *params, const void *points,
                                 const int32_t *n_valid, const int8_t *charge, int64_t S,
                                 const int64_t *seed_index, const void *wires, int32_t W,
                                 int32_t ldw, const int32_t *hit_offsets, const void *drift,
                                 uint8_t *hit_mask, uint8_t *hit_class, void *dca_wire,
                                 int32_t update_mask, comet_stream stream);

#ifdef __cplusplus
}
#endif

#endif /* COMET_SCAN_H */
