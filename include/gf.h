/*
 * gf.h -- C ABI of libgf: SU(3) Landau / Coulomb gauge fixing by checkerboard
 * overrelaxation on one NVIDIA GB300 (sm_103a).
 *
 * Method: N. Cardoso, "Coulomb and Landau Gauge Fixing in GPUs using CUDA and MILC"
 * (Lattice 2014).  The gauge condition is the maximum of the functional F_U[g] of
 * Eq. (1); its quality is theta of Eqs. (2)-(3); the overrelaxation algorithm is
 * Algorithm 1 with the local SU(2)-subgroup maximisation of Eqs. (4)-(6).
 *
 * Conventions used by every call
 * -------------------------------
 *  - dims = {Lx, Ly, Lz, Lt}; every extent even and >= 2 (Section 2 requires even local
 *    extents for the checkerboard); direction mu = 0, 1, 2, 3 is x, y, z, t (time is
 *    mu = 3, Section 1).  Periodic boundaries in every direction.
 *  - Canonical field layout (host or device buffers passed to upload/download):
 *    interleaved (re, im) float64 pairs of a complex array of shape
 *    (Lt, Lz, Ly, Lx, 4, 3, 3), row-major, x fastest: link U_mu(x) of site
 *    s = x + Lx*(y + Ly*(z + Lz*t)) starts at element 2*9*(4*s + mu).
 *  - Site parity p(x) = (x + y + z + t) mod 2; parity 0 ("even") is updated first.
 *  - Landau gauge uses nd = 4 directions in K(x), F and Delta(x); Coulomb gauge uses
 *    nd = 3 (the temporal links are still transformed: Algorithm 1 updates every mu).
 *    F is normalised by 1/(nd * 3 * V) so that the unit field has F = 1.
 *  - A handle holds one lattice (gf_create) or a batch of independent lattices
 *    (gf_create_batch).  Convergence units: one per lattice for Landau gauge, one per
 *    (lattice, time slice) for Coulomb gauge; each unit has its own stop rule and mask.
 *  - Streams: every call enqueues work on the CUDA stream given at creation (NULL =
 *    legacy default stream).  Calls that return host values synchronise that stream.
 *  - Memory: the caller may pass a device workspace of at least gf_workspace_bytes()
 *    bytes (e.g. a framework's caching allocator); the handle then allocates no device
 *    memory of its own.  With workspace == NULL the handle allocates it with cudaMalloc
 *    and frees it in gf_destroy.  The caller keeps ownership of every buffer it passes.
 *  - Errors: every int-returning call returns GF_OK (0) on success, a negative GF_E*
 *    code on failure (nothing is left half-done on the host; device work already
 *    enqueued may have run), or GF_ENOTCONVERGED (positive, not a failure).  No C++
 *    exception crosses this interface.  gf_last_error() gives a readable message.
 *  - Handles are not thread-safe: one host thread at a time per handle.
 */
#ifndef GF_H
#define GF_H

#include <stddef.h>

#if defined(__GNUC__)
#define GF_API __attribute__((visibility("default")))
#else
#define GF_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define GF_OK 0
#define GF_ENOTCONVERGED 1 /* gf_fix stopped at maxiter with a unit still above eps */
#define GF_EINVAL (-1)     /* bad argument: dims, enum, null pointer, size */
#define GF_ECUDA (-2)      /* a CUDA runtime call failed; see gf_last_error */
#define GF_ENOMEM (-3)     /* workspace too small or device allocation failed */
#define GF_ESTATE (-4)     /* call not valid in the handle's current state */

/* gauge condition (Section 1, Eq. (3) and the sentence after it) */
#define GF_LANDAU 0
#define GF_COULOMB 1

/* link storage in device memory (Section 2: 18, 12 or 8 real numbers per SU(3) link) */
#define GF_FP64_18 0 /* full matrix, FP64 */
#define GF_FP32_18 1 /* full matrix, FP32 */
#define GF_FP32_12 2 /* rows 0 and 1, FP32; row 2 = conj(row0 x row1) on every load */
#define GF_FP64_12 3 /* rows 0 and 1, FP64; row 2 rebuilt on every load */
#define GF_FP32_8 4  /* u01, u02, u10, arg u00, arg u20 in FP32; rows 0 and 1 rebuilt from
                        unitarity on every load (divides by N = |u01|^2 + |u02|^2: links with
                        N = 0 keep only their row 0, the 2x2 block becomes e^{-i arg(u00)/2} 1) */
#define GF_FP64_8 5  /* the same 8 reals in FP64 */

/* creation flags */
#define GF_FLAG_MIXED 1 /* keep a polish copy (144 bytes per link): gf_fix runs the FP32
                           storage down to the switch threshold, converts, then polishes
                           (double-float, then FP64; see gf_set_polish) (ignored for the
                           FP64 storages) */
#define GF_FLAG_AUTOGRAD 4 /* add the buffers of gf_ad_functional / gf_ad_backward (one
                              lattice, GF_FP64_18) */
#define GF_FLAG_FASD 2  /* add the buffers of Fourier-accelerated steepest descent (one
                           lattice; GF_FP32_12 or GF_FP64_18; power-of-two extents <= 64 in
                           the transformed directions: x, y, z, and t for Landau gauge) */

/* form of the overrelaxation g -> g^omega per SU(2) subgroup (Section 1, after Eq. (6)) */
#define GF_OR_FIRST_ORDER 0 /* a' = 1 - omega + omega a, b' = omega b, renormalised */
#define GF_OR_EXACT 1       /* exact SU(2) power of the subgroup maximiser */

typedef struct gf_handle gf_handle;

/*
 * Bytes of device workspace a handle needs.
 *   n_lat: number of lattices (1 for gf_create); dims: n_lat * 4 ints as above;
 *   gauge: GF_LANDAU | GF_COULOMB; storage: one of the GF_FP* codes above;
 *   flags: 0 or a combination of GF_FLAG_* (GF_FLAG_MIXED for the FP32 storages).
 *   *bytes receives the size.  Host-only (no CUDA call).  Returns GF_EINVAL on bad
 *   arguments.
 */
GF_API int gf_workspace_bytes(int n_lat, const int *dims, int gauge, int storage, int flags,
                       size_t *bytes);

/*
 * Create a handle for one lattice (Section 1 problem statement; Eq. (1) with Nc = 3).
 *   dims: {Lx, Ly, Lz, Lt}, even, >= 2.  nc: must be 3 (GF_EINVAL otherwise).
 *   stream: a cudaStream_t (or NULL).  workspace / workspace_bytes: caller-owned device
 *   memory (16-byte aligned, >= gf_workspace_bytes) or NULL / 0.
 *   *out receives the handle; on failure *out is NULL.  The links start undefined:
 *   call gf_upload before sweeping.
 */
GF_API int gf_create(const int dims[4], int nc, int gauge, int storage, int flags, void *stream,
              void *workspace, size_t workspace_bytes, gf_handle **out);

/*
 * Create a handle for n_lat independent lattices of possibly different extents (a batch
 * of configurations fixed together: one launch per half-sweep covers all of them).
 *   dims: n_lat * 4 ints.  Other arguments as gf_create.
 */
GF_API int gf_create_batch(int n_lat, const int *dims, int gauge, int storage, int flags,
                    void *stream, void *workspace, size_t workspace_bytes, gf_handle **out);

/* Release the handle (and the workspace, if the handle allocated it).  NULL is a no-op. */
GF_API void gf_destroy(gf_handle *h);

/* Message of the last failure on this handle ("" if none); h == NULL gives the message of
   the last failed gf_workspace_bytes / gf_create / gf_create_batch /
   gf_functional_theta_noalloc on this thread.  Valid until the next call. */
GF_API const char *gf_last_error(const gf_handle *h);

/* Number of lattices and of convergence units (see conventions). */
GF_API int gf_num_lattices(const gf_handle *h);
GF_API int gf_num_units(const gf_handle *h);

/*
 * Copy lattice `lat` of the batch in (upload) or out (download), converting between the
 * canonical layout and the internal structure-of-arrays layout (Section 2: parity-split
 * sites, each complex element of a link at a stride of 4 V).
 *   links: canonical layout, 2*9*4*V float64; on_device = 1 if it is device memory,
 *   0 if host memory (pinned memory gives the fastest copies).
 *   Upload rounds to the handle's storage (FP32 and/or 12 or 8 reals: the other
 *   elements are dropped) and resets the sweep count (gf_get_sweeps_done), the masks
 *   (all units active) and the iteration counts.  Download rebuilds the dropped
 *   elements (rows 0, 1 of 8-real storage in the storage's precision, row 2 in FP64).
 *   In mixed mode gf_fix leaves the field in the FP64 copy and download reads that copy;
 *   an upload moves the handle back to its primary storage, so upload every lattice of
 *   a batch before the next gf_fix.  Device buffers must be 16-byte aligned.  Both
 *   calls synchronise the stream when on_device = 0 (the host buffer is complete on
 *   return).
 */
GF_API int gf_upload(gf_handle *h, int lat, const double *links, int on_device);
GF_API int gf_download(gf_handle *h, int lat, double *links, int on_device);

/*
 * F (Eq. (1), in-place links so g = 1) and theta (Eqs. (2)-(3)) of the current field.
 *   F, theta: n_lat entries each (nullable).  unit_F, unit_theta: gf_num_units entries
 *   each (nullable); for Coulomb gauge unit (lat, t) has F_t and theta_t normalised by
 *   the slice volume.  Sums are accumulated in FP64 in a fixed order (bit-reproducible
 *   for a given handle).  Synchronises the stream.
 */
GF_API int gf_functional_theta(gf_handle *h, double *F, double *theta, double *unit_F,
                        double *unit_theta);

/*
 * One checkerboard half-sweep (parity 0 or 1) or a full sweep (parity 2 = even then
 * odd) of Algorithm 1 over all active units, with overrelaxation parameter omega in
 * [1, 2) (Section 1, after Eq. (6)).  Per site: K(x) of Eq. (5) in place, the three
 * SU(2)-subgroup maximisers (0,1), (0,2), (1,2) with g -> g^omega, and g(x) applied
 * to U_mu(x) and U_mu(x - mu) for all four mu.  Asynchronous; no reunitarisation.
 */
GF_API int gf_or_sweep(gf_handle *h, int parity, double omega);

/* Project every link of the current field back to SU(3) (Gram-Schmidt on rows 0, 1;
   row 2 = conj(row0 x row1)), as done every 20 sweeps in Section 3.  Asynchronous. */
GF_API int gf_reunitarize(gf_handle *h);

/*
 * Algorithm 1: measure; while a unit has theta >= eps and fewer than maxiter sweeps
 * were done: even half-sweep, odd half-sweep (reunitarising the links it writes after
 * every reunit_interval-th sweep), then the stop check every check_interval sweeps; a
 * unit whose theta < eps is masked and no longer updated.  The check forms F and the
 * odd-site part of theta inside the odd half-sweep; theta >= that part, so a unit whose
 * odd part alone reaches eps continues exactly as the full theta would decide, and the
 * even-site part is computed only for the other units and on the last sweep of the
 * budget.  The measurement before the first sweep follows the same rule: the odd-site
 * pass decides every unit whose odd part reaches eps, and the even-site pass runs only
 * if some unit is undecided (a field already below eps returns the values
 * gf_functional_theta gives).  F, theta and the masks at exit are exact
 * (gf_set_history records theta at every check).  FP32 storages take the odd-site values from K' = G K (K of Eq. (5)
 * before the site's update, G its new transformation: Delta of the updated links is the
 * traceless anti-Hermitian part of K', Re Tr K' the site's share of Eq. (1)), i.e. of the
 * links before a reunitarisation in the same sweep, a difference at the rounding level;
 * FP64 and the double-float polish sum the stored links.  The schedule counts sweeps
 * from the last upload (gf_get_sweeps_done).
 *   eps > 0; maxiter >= 0.  iters (nullable): gf_num_units ints, sweeps each unit
 *   received.  F, theta (nullable): n_lat final values.
 *   With GF_FLAG_MIXED each lattice has its own precision level: FP32 sweeps until all
 *   its units have theta < the switch threshold (gf_set_mixed_switch, default 1e-8),
 *   then its links are converted (with an FP64 reunitarisation) to the polish
 *   (gf_set_polish), whose sweeps run until its units have theta < eps, and finally to
 *   FP64-18, where theta is measured again and FP64 sweeps continue until it is below
 *   eps.  Lattices of a batch move on independently (a unit below its level's threshold
 *   waits for the other units of its lattice: the time slices of a Coulomb lattice share
 *   its temporal links and change precision together); a moved lattice is measured at
 *   its new level before it sweeps.  One launch per half-sweep and level covers every
 *   lattice at that level; a lattice that becomes ready in the middle of a CUDA-graph
 *   replay of 16 sweeps moves at the end of that replay.  At exit every lattice is in
 *   the FP64 copy (download and gf_functional_theta read it).  iters counts a unit's
 *   sweeps at every level; maxiter bounds the sweeps of the whole call, whose
 *   reunitarisation and check schedules count from 0.  Returns GF_OK when every unit
 *   converged, GF_ENOTCONVERGED at maxiter.  Synchronises the stream.
 */
GF_API int gf_fix(gf_handle *h, double eps, int maxiter, int *iters, double *F, double *theta);

/*
 * Fourier-accelerated steepest descent, Algorithm 2 with Eqs. (7)-(9): one iteration
 *   Delta(x) (Eq. (3), the argument of Eq. (8)); FFT of each element over the gauge
 *   directions (4D Landau, 3D per time slice Coulomb); multiply by
 *   (alpha/2) p^2_max / p^2, p^2 = sum_mu 4 sin^2(pi k_mu / L_mu), p^2_max = 4 nd, the
 *   k = 0 mode set to 0; inverse FFT and 1/N; g(x) = reunit(1 + Delta~(x)) (first-order
 *   exponential); U_mu(x) <- g(x) U_mu(x) g(x+mu)^+ for every mu.
 * Needs a handle created with GF_FLAG_FASD.  Asynchronous.  alpha > 0 (0.08 in the paper,
 * Sec. 1).  gf_fix runs Algorithm 2 instead of Algorithm 1 after
 * gf_set_method(h, GF_METHOD_FASD), with gf_set_alpha's alpha [0.08] and the links
 * reunitarised every reunit_interval iterations; in Coulomb gauge each time slice has
 * its own stop rule.  Mixed precision does not apply to it.
 */
#define GF_METHOD_OR 0
#define GF_METHOD_FASD 1
GF_API int gf_fa_sd_step(gf_handle *h, double alpha);
GF_API int gf_set_method(gf_handle *h, int method);
GF_API int gf_set_alpha(gf_handle *h, double alpha);

/*
 * F and theta as differentiable functions of the gauge transformation's Lie-algebra
 * parameters (the gradient direction of steepest descent, Eq. (7)):
 *   g(x) = exp(i sum_a c_a(x) lambda_a) (Gell-Mann lambda_a), U^g_mu(x) = g(x) U_mu(x)
 *   g(x+mu)^+ applied to the handle's current field, F(c) by Eq. (1) and theta(c) by
 *   Eqs. (2)-(3) of U^g.
 * gf_ad_functional: c = device array of V x 8 doubles in canonical site order; out =
 *   device array of 2 doubles, receives (F, theta).
 * gf_ad_backward: upstream = device (dL/dF, dL/dtheta); grad = device V x 8 doubles,
 *   overwritten with dL/dc.  g, the transformed links and Delta are recomputed from c
 *   (nothing is kept from the forward call).  dF/dc_a(x) at c = 0 is
 *   Tr[lambda_a Delta(x)] / (2i nd Nc V).
 * Both asynchronous on the handle's stream; the handle needs GF_FLAG_AUTOGRAD.
 */
GF_API int gf_ad_functional(gf_handle *h, const double *c, double *out);
GF_API int gf_ad_backward(gf_handle *h, const double *c, const double *upstream, double *grad);

/* Settings (defaults in brackets).  Each returns GF_EINVAL for an out-of-range value. */
GF_API int gf_set_omega(gf_handle *h, double omega);          /* [1.7], 1 <= omega < 2       */
GF_API int gf_set_overrelax_form(gf_handle *h, int form);     /* [GF_OR_FIRST_ORDER]          */
GF_API int gf_set_reunit_interval(gf_handle *h, int n);       /* [20], 0 = never              */
GF_API int gf_set_check_interval(gf_handle *h, int n);        /* [1], >= 1                    */
GF_API int gf_set_mixed_switch(gf_handle *h, double eps_sw);  /* [1e-8], > 0                  */
GF_API int gf_set_reproducible(gf_handle *h, int on);         /* [0]; 1 = FP64-18 sweeps without
                                  fused multiply-add and with IEEE divisions, in the
                                  oracle's operation order (bit-reproducible results);
                                  no effect on the other storages */
GF_API int gf_set_block_size(gf_handle *h, int threads);      /* [128]; 64, 128 or 256        */

/* Half-sweep kernel for FP32-12 storage: GF_SWEEP_REGISTER holds each site's 8 links in
   registers; GF_SWEEP_PIPELINED stages them through shared memory with asynchronous
   copies one tile ahead (persistent CTAs).  Both give the same results.  AUTO [default]
   = PIPELINED for FP32-12; other storages always use the register kernel, and asking
   them for PIPELINED returns GF_EINVAL. */
/* Arithmetic of the polish phase of a mixed-precision gf_fix (GF_FLAG_MIXED):
   GF_POLISH_SPLIT [default]: double-float sweeps (each real an unevaluated sum of two
   floats, about 48-bit precision, no FP64 arithmetic in the sweep) with the first-order
   overrelaxation form, then conversion to FP64-18 with an FP64 reunitarisation and
   FP64 sweeps until theta, measured in FP64, is below eps.  The polish sweep moves 3x
   the bytes of an FP32-12 sweep at the memory bandwidth, where an FP64-18 sweep is
   bound by the FP64 pipe (about 7x slower on this GPU), so this is the default.  With
   GF_OR_EXACT the FP64 polish is used.
   GF_POLISH_FP64: FP64-18 sweeps straight after the FP32 phase. */
#define GF_POLISH_FP64 0
#define GF_POLISH_SPLIT 1
GF_API int gf_set_polish(gf_handle *h, int polish);

#define GF_SWEEP_AUTO 0
#define GF_SWEEP_REGISTER 1
#define GF_SWEEP_PIPELINED 2
GF_API int gf_set_sweep_variant(gf_handle *h, int variant);

/* Autotuner: times 7 sweeps (2 warm-up) of the current field for each block size (64,
   128, 256) and sweep kernel (register / pipelined for FP32-12) with CUDA events on the
   handle's stream and keeps the fastest; *threads_out, *variant_out (nullable) receive
   the choice.  The timing sweeps are applied to the field (they are gauge
   transformations of it): tune before uploading the field to fix, or upload it again
   afterwards.  Synchronises the stream. */
GF_API int gf_autotune(gf_handle *h, int *threads_out, int *variant_out);

/* Checkpoint / resume.  The handle counts the sweeps (or Fourier-accelerated iterations)
   done since the last upload; the reunitarisation and check schedule of gf_fix continues
   from that count (the sweep after n sweeps is sweep n + 1).  To resume a run: download
   the links, read the count, later upload the links into a handle with the same settings
   and set the count; the continued run gives the bits of the uninterrupted one (FP64-18,
   or any storage in non-mixed mode).  Mixed-precision gf_fix counts from 0 over all its
   precision levels and leaves the count at the sweeps it did.  Upload resets it to 0. */
GF_API int gf_get_sweeps_done(const gf_handle *h, int *n);
GF_API int gf_set_sweeps_done(gf_handle *h, int n);

/* Sweeps of the last gf_fix in which some unit swept at FP32 precision, and in which some
   unit swept at a polish precision (double-float or FP64), nullable.  With one lattice the
   two phases follow each other and add up to its sweeps; in a batch they can overlap. */
GF_API int gf_fix_phase_sweeps(const gf_handle *h, int *fp32_sweeps, int *fp64_sweeps);

/*
 * Convergence history of gf_fix (Algorithm 1 computes theta after every sweep).
 *   buf: device memory (or host memory mapped for the device) for `capacity` records of
 *   1 + 2 * n_lat doubles: the sweep number within the gf_fix call (0 = the field before
 *   the first sweep), then F and theta of every lattice (Eqs. (1)-(3); for Coulomb gauge
 *   the totals over the slices).  One record per check sweep (gf_set_check_interval);
 *   records beyond `capacity` are dropped.  While a history is set every check measures
 *   theta in full (the loop otherwise skips the even-site part where the odd-site part
 *   alone decides the stop), so sweeps are slower.  capacity = 0 (or buf = NULL with
 *   capacity 0) turns it off.  The caller owns buf and keeps it alive while it is set.
 *   Overrelaxation only (not the Fourier-accelerated loop).
 *   gf_history_count: records written by the last gf_fix.
 */
GF_API int gf_set_history(gf_handle *h, double *buf, int capacity);
GF_API int gf_history_count(const gf_handle *h, int *n);

/*
 * F and theta of a field held in device memory, with no allocation of any kind.
 *
 * The paper has no counterpart to this call; it exists for callers that cannot
 * allocate device memory: code that runs inside a memory pool reserved up front by a
 * framework, a loop that must not call cudaMalloc because it may synchronise the
 * device, or a host process whose device allocations all belong to someone else.
 * Such a caller passes only its input and output buffers and gets the values of
 * gf_functional_theta without a handle or a workspace.
 *   dims: {Lx, Ly, Lz, Lt}, even, >= 2, at most GF_NOALLOC_MAX_BLOCKS * 256 sites in
 *   all (larger lattices return GF_EINVAL with a message saying so).
 *   gauge: GF_LANDAU or GF_COULOMB.  links: device memory, canonical layout (as for
 *   gf_upload), 16-byte aligned.  out: device memory for 2 doubles, receives F and
 *   theta.  stream: cudaStream_t (NULL = legacy default stream); the call is
 *   asynchronous on it.
 * Its block partial sums live in one static device array of
 * (32 + 2 * GF_NOALLOC_MAX_BLOCKS) doubles (about 4 MiB) that every GPU loading this
 * library holds until the process exits.  All calls share that array: calls that
 * overlap on the GPU (different streams or host threads) race on it and give wrong
 * results; calls on one stream are safe.  The first call on each device looks up the
 * array's device address with that device current, so make that first call before any
 * stream capture.  The address is kept for the life of the process: a device reset
 * (cudaDeviceReset, or the primary context torn down and created again) between calls
 * is not supported.  The extents are checked before any CUDA call, with an overflow-free
 * volume, so no input reaches the kernel with more sites than the array covers.
 * Errors: GF_EINVAL / GF_ECUDA, message in gf_last_error(NULL).
 */
#define GF_NOALLOC_MAX_BLOCKS 262144
GF_API int gf_functional_theta_noalloc(const int dims[4], int gauge, const double *links,
                                       double *out, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* GF_H */
