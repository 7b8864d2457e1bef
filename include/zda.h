/*
 * zda.h -- C ABI of libzda: the GPU zone solver of the zoned discrete
 * axisymmetry (ZDA) metalens method (arXiv 2501.07979).
 *
 * One call family per step of the method:
 *   zone geometry ............ section "Zoned discrete axisymmetry (ZDA)",
 *                              Eqs. 1-2 (n-fold wedge, tau = 2 pi / n)
 *   Yee time loop ............ section "Differentiable FDTD in cylindrical
 *                              coordinates", Eqs. 3-5 (Bloch-reduced curl,
 *                              stretched-coordinate PMLs in r and z)
 *   density -> permittivity .. Eq. 6 plus the conic and binarisation filters
 *                              ("Results and Discussion")
 *   focal intensity .......... "Results and Discussion" (focal-spot far-field
 *                              intensity of a normally incident plane wave,
 *                              m = +-1) and Eq. 9's focal intensity I
 *   adjoint gradient ......... section "Differentiable FDTD": hybrid
 *                              time/frequency adjoint, all frequencies from
 *                              one forward and one adjoint run
 *
 * Units: c = eps0 = mu0 = 1 and lambda0 = 1 (lengths in lambda0, times in
 * lambda0 / c).
 *
 * Conventions for every call:
 *  - Pointers named *_dev are device pointers (e.g. from torch tensors) on
 *    the zone's device; pointers named *_host (or documented as host) are
 *    host memory.  The caller owns all memory it passes; the library never
 *    frees or retains caller memory past the call, except the workspace
 *    bound with zda_zone_bind_workspace, which it uses until the zone is
 *    destroyed or another workspace is bound.
 *  - The library allocates no device memory of its own.
 *  - `stream` is a cudaStream_t (NULL = legacy default stream).  Device work
 *    is enqueued on it.  Calls that return host results (zda_forward's
 *    focal_out, zda_iteration's outputs) synchronise that stream before
 *    returning; others return once the work is enqueued.
 *  - Every call returns a zda_status; nothing aborts, traps or exits.  On
 *    error, zda_last_error() returns a message for the calling thread.
 *  - Complex arrays are interleaved (re, im) floats or doubles.
 *  - A zone object is not thread-safe; calls on one zone must not overlap.
 */
#ifndef ZDA_H
#define ZDA_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    ZDA_OK = 0,
    ZDA_ERR_ARG = -1,        /* invalid argument or descriptor */
    ZDA_ERR_CUDA = -2,       /* a CUDA runtime call failed */
    ZDA_ERR_OOM = -3,        /* workspace too small / host allocation failed */
    ZDA_ERR_TIMEOUT = -4,    /* a bounded device-side wait gave up */
    ZDA_ERR_NONFINITE = -5,  /* NaN or Inf in the focal phasors (solver blew up) */
    ZDA_ERR_STATE = -6       /* call out of order (e.g. adjoint before forward) */
} zda_status;

#define ZDA_MAX_LAYERS 8
#define ZDA_MAX_FREQ 16      /* signed frequencies = 2 x wavelengths */
#define ZDA_MAX_FILTER_TAPS 65536   /* conic-filter taps per pixel, (2 di + 1)(2 dj + 1) */

typedef struct zda_ctx zda_ctx;
typedef struct zda_zone zda_zone;
typedef struct zda_lens zda_lens;

/* Zone descriptor (plain data, copied at zda_zone_create).
 * n_fold = 0 selects continuous axisymmetry (the axis zone, section "Centimeter-
 * scale metalens": the first zone is continuously axisymmetric): n_phi = 1,
 * every (1/r) d/dphi is i m / r, r_lo >= 0 (r_lo = 0 puts the axis inside,
 * then pml_r_in = 0); dt uses (m / max(r_lo, dr/2))^2 for the azimuthal term.
 * The simulated domain is r in [r_lo, r_lo + n_r dr], one wedge
 * phi in [0, 2 pi / n_fold) with n_phi cells (Bloch-periodic with phase
 * e^{i m 2pi/n_fold}), z in [0, n_z dz].  pml_* cells of CPML line the r and
 * z ends (PEC behind them).  The design / monitor annulus is
 * r in [r_lo + pml_r_in dr, r_lo + (n_r - pml_r_out) dr].
 * Layer l (permittivity layer_eps[l]) covers z-cells k >= layer_k0[l] up to
 * the next layer's start; z-cells [design_k0, design_k1) are the design layer
 * with eps = eps_lo + rho~ (eps_hi - eps_lo) over the design annulus (Eq. 6)
 * and eps_lo inside the r-PMLs.  The plane-wave source sheet sits on the
 * E_r/E_phi plane source_k, the monitor on plane monitor_k (both above the
 * z-PML).  dt = courant / sqrt(1/dr^2 + 1/(r_lo dphi)^2 + 1/dz^2).
 * filter_radius <= 0 disables the conic filter, beta <= 0 the projection.
 * The filter spans di = min(floor(R / dr), n_r_design - 1) radial and
 * dj = floor(R / (r_c dphi)) azimuthal neighbours (r_c: the first design
 * row's radius); a radius with (2 di + 1)(2 dj + 1) > ZDA_MAX_FILTER_TAPS is
 * refused (ZDA_ERR_ARG).
 * focal is the focal distance above the top of the design layer. */
typedef struct {
    double r_lo, dr, dz;
    int n_r, n_phi, n_z;
    int n_fold, m;
    int pml_r_in, pml_r_out, pml_z;
    int n_layers;
    int layer_k0[ZDA_MAX_LAYERS];
    double layer_eps[ZDA_MAX_LAYERS];
    int design_k0, design_k1;
    double eps_lo, eps_hi;
    int source_k, monitor_k;
    double courant;
    int n_steps;
    double filter_radius, beta, eta;
    double focal;
} zda_zone_desc;

/* Derived sizes and layouts, filled by zda_zone_query. */
typedef struct {
    double dt, dphi, tau;
    int n_freq;            /* 2 x wavelengths: +w_0..+w_{L-1}, -w_0..-w_{L-1} */
    int n_r_design;        /* n_r - pml_r_in - pml_r_out */
    int design_nk;         /* design_k1 - design_k0 + 1 E planes in the DFT box */
    size_t workspace_bytes;
    long long cells;       /* n_r n_phi n_z */
} zda_zone_info;

/* Library context bound to one CUDA device (cudaSetDevice is called by the
 * library on entry to every call that takes a ctx or zone). */
zda_status zda_ctx_create(zda_ctx **out, int device);
void zda_ctx_destroy(zda_ctx *ctx);

/* Create a zone (validates the descriptor, computes the FP64 host tables of
 * the geometry).  Wavelengths default to {1.0}; pulse to f0 = 1,
 * sigma_t = 0.5, t0 = 2. */
zda_status zda_zone_create(zda_ctx *ctx, const zda_zone_desc *desc, zda_zone **out);
void zda_zone_destroy(zda_zone *zone);

/* Design wavelengths (lambda0 units), 1 <= n_lambda <= ZDA_MAX_FREQ/2.  The
 * signed frequency list is +2pi/lambda_l then -2pi/lambda_l (the m = +1 run
 * carries the m = -1 field as its conjugate at -w). */
zda_status zda_set_wavelengths(zda_zone *zone, const double *lambda_host, int n_lambda);

/* Source pulse g(t) = cos(2 pi f0 (t - t0)) exp(-(t - t0)^2 / (2 sigma_t^2)). */
zda_status zda_set_pulse(zda_zone *zone, double f0, double sigma_t, double t0);

/* Binarisation strength of the tanh projection for the next runs (the
 * continuation of beta during a topology optimisation, "Results and
 * Discussion"): beta <= 0 turns it off, 0 < eta < 1. */
zda_status zda_zone_set_projection(zda_zone *zone, double beta, double eta);

/* Sizes / layouts (workspace_bytes depends on wavelengths and n_steps). */
zda_status zda_zone_query(const zda_zone *zone, zda_zone_info *info);
zda_status zda_zone_workspace_bytes(const zda_zone *zone, size_t *bytes);

/* Bind caller-allocated device memory (>= workspace_bytes, 256-byte aligned)
 * as the zone's workspace: fields, CPML auxiliaries, DFT accumulators and
 * tables.  Re-bind after changing wavelengths or n_steps. */
zda_status zda_zone_bind_workspace(zda_zone *zone, void *workspace_dev, size_t bytes);

/* Forward solve (one FDTD run): rho_dev [n_r_design][n_phi] floats in [0,1]
 * at the (r, phi) design-pixel centres -> conic filter -> projection ->
 * Eq. 6 eps -> n_steps Yee steps with the m = +1 plane-wave source and
 * running DFTs (monitor plane and design volume) -> on-axis focal phasors.
 * focal_out_host: n_freq complex doubles S_q (interleaved), q in the signed
 * frequency order; the focal intensity is I = 2 sum_q |S_q|^2.  Keeps the
 * forward DFTs in the workspace for zda_adjoint. */
zda_status zda_forward(zda_zone *zone, const float *rho_dev, double *focal_out_host, void *stream);

/* Adjoint run (second FDTD run) and gradient: dI_dfocal_host holds n_freq
 * complex doubles (dI/dRe S_q, dI/dIm S_q) for any real objective I(S);
 * grad_rho_dev [n_r_design][n_phi] floats receives dI/drho.  Requires a
 * preceding zda_forward with the same rho (ZDA_ERR_STATE otherwise).  With
 * the fused step it synchronises the stream to report wait timeouts. */
zda_status zda_adjoint(zda_zone *zone, const double *dI_dfocal_host, float *grad_rho_dev, void *stream);

/* One TopOpt iteration of the summed focal intensity I = 2 sum |S_q|^2:
 * forward, dI/dS = 4 S, adjoint.  host_buffers != 0: rho and grad_rho are
 * HOST pointers and the call copies them to / from the workspace on
 * `stream`; otherwise they are device pointers.  I_out_host: 1 double. */
zda_status zda_iteration(zda_zone *zone, const float *rho, double *I_out_host, float *grad_rho,
                         int host_buffers, void *stream);

/* Step-level entry points (each step of the path on its own). */

/* Conic filter + tanh projection: rho_dev -> rho_tilde_dev (both
 * [n_r_design][n_phi]). */
zda_status zda_filter_project(zda_zone *zone, const float *rho_dev, float *rho_tilde_dev, void *stream);

/* Transposed chain: given rho_dev (the forward input) and g_tilde_dev =
 * dI/drho~, write dI/drho = F^T (P'(F rho) g_tilde) to grad_rho_dev. */
zda_status zda_filter_project_backward(zda_zone *zone, const float *rho_dev, const float *g_tilde_dev,
                                       float *grad_rho_dev, void *stream);

/* On-axis near-to-far transform of a monitor-plane DFT given by the caller:
 * monitor_dft_dev complex floats [n_freq][2][n_r][n_phi] (E_r, E_phi sites)
 * -> focal_out_host n_freq complex doubles (synchronises the stream). */
zda_status zda_focal_transform(zda_zone *zone, const float *monitor_dft_dev, double *focal_out_host,
                               void *stream);

/* The focal transform evaluated on the zone surrogate's output (zda_nn.h):
 * y_dev [n][n_r_design][n_phi][4 Q] (device FP32) holds the monitor DFT of
 * the design rows, channel (q 2 + comp) 2 + part (comp 0 = E_r, 1 = E_phi;
 * part 0 = real, 1 = imaginary) divided by `scale`.  Writes the focal
 * phasors S_dev [n][Q] (device, interleaved complex FP64) of "Results and
 * Discussion" restricted to those rows (the outer-edge E_phi node, weight
 * dr / 2, is not among them).  The _transpose call is its transpose: from
 * dS_dev [n][Q] (dobj/dRe S + i dobj/dIm S, device) it writes
 * dobj/dy [n][n_r_design][n_phi][4 Q] to dy_dev.  Needs a zone (no run). */
zda_status zda_focal_transform_nn(zda_zone *zone, const float *y_dev, int n, float scale, double *S_dev, void *stream);
zda_status zda_focal_transform_nn_transpose(zda_zone *zone, const double *dS_dev, int n, float scale, float *dy_dev,
                                    void *stream);

/* Copies of internal state after zda_forward / zda_adjoint (complex floats):
 *   zda_copy_fields:  [6][n_r][n_phi][n_z]  E_r, E_phi, E_z, H_r, H_phi, H_z
 *   zda_copy_monitor_dft: [n_freq][2][n_r][n_phi]
 *   zda_copy_design_dft:  [n_freq][3][n_r][n_phi][design_nk]; which = 0
 *                         forward run, 1 adjoint run. */
zda_status zda_copy_fields(zda_zone *zone, float *out_dev, void *stream);
zda_status zda_copy_monitor_dft(zda_zone *zone, float *out_dev, void *stream);
zda_status zda_copy_design_dft(zda_zone *zone, int which, float *out_dev, void *stream);

/* Number of kernel launches the library issued since the zone was created
 * (for launch accounting in benchmarks). */
long long zda_zone_launch_count(const zda_zone *zone);

/* Time-step kernel of the zone (Eqs. 3-4 advanced one step).  variant 0:
 * two launches per step (H update, E update), in place, two z-cells per
 * thread with 16-byte loads when n_z and pml_z are even (wedge zones), else
 * one z-cell per thread; tile_phi in {4, 8, 16, 32} is the thread block's
 * phi rows (256 threads; other values: 4 for zones of at most 16 phi cells,
 * else 16), i_ranges = 3 runs the E update at 3 thread blocks per SM (fewer
 * registers, a few spilled), else 2.  variant 2: the same with one z-cell
 * per thread always.  variant 4 (annular zones, even n_z and pml_z,
 * real-radius r-PML): the split step with its E update on tiles of tile_phi
 * in {8, 16, 32} phi rows x 32 z-cells whose H and E values are staged into
 * shared memory by TMA tensor copies several radii ahead, each thread block
 * streaming over one of i_ranges radius ranges (0 = radius ranges of about
 * 21 radii).  variant 5 (as variant 4): both halves of the split step on
 * those tiles (the H update stages E^n of two radii and H^{n-1/2}).
 * variant 1 (annular zones, n_z <= 256): one fused launch per
 * step (E and H updated together, ping-pong field buffers, streaming along
 * r; tile_phi in {2, 4} phi rows per thread block, i_ranges radius ranges
 * per phi tile, 0 = as many as fit in one wave).  variant 3 (annular zones,
 * even n_z and pml_z, real-radius r-PML): one fused launch per step on
 * tiles of tile_phi in {4, 8, 16} phi rows x 32 z-cells staged by TMA, each
 * thread block streaming over one of i_ranges radius ranges (0 = about 21
 * radii each).  Default at zone creation: variant 4 with 16 rows where it
 * applies and the zone gives at least four waves of its thread blocks (2 per
 * SM) in radius ranges of about 21 radii, else variant 0; selecting
 * the stretched r-PML (form 1) on a zone that still has the default falls
 * back to variant 0, while an explicit variant 1, 3 or 4 refuses it.  All
 * compute the same scheme; results agree to FP32 rounding.  Variants 1, 3
 * and 4 bound their device-side waits (zda_zone_set_wait_limit). */
zda_status zda_zone_set_kernel(zda_zone *zone, int variant, int tile_phi, int i_ranges);
zda_status zda_zone_get_kernel(const zda_zone *zone, int *variant, int *tile_phi, int *i_ranges);

/* Form of the radial PML ("Differentiable FDTD in cylindrical coordinates":
 * the stretched coordinate r' = r + i zeta_r(r) / w appears explicitly in the
 * equations, and the r-PML has to be regularised).
 * form 0 (default): convolutional PML on every d/dr term, the whole
 *   (1/r) d/dr (r .) of the z-curls stretched, real radius in every metric
 *   factor.
 * form 1: stretched coordinates.  Inside the r-PML the z-curls are
 *   (1/s_r) dF/dr + X / r~ with the metric part X = (F(i+1) + F(i)) / 2 -+
 *   dG/dphi, and the r-curls take (1/r~) dG/dphi; in the outer slab r~ = r + Omega / (alpha - i w),
 *   Omega = int sigma dr' (alpha constant over the slab, so dr~/dr = s_r),
 *   realised as one more recursive convolution per H_r, H_z, E_r, E_z site.
 *   The inner slab keeps r~ = r (the regularisation: with the stretched inner
 *   radius Im r~ < 0 and the wedge's non-propagating azimuthal orders grow).
 *   Reflection of a cylindrical pulse at w0, against a radially larger
 *   domain: 1.9e-3 (form 0) vs 5e-5 (form 1) at r = 10 lambda.
 * Form 1 runs on the split step (variants 0 and 2); the fused steps
 * (variants 1 and 3) refuse it (ZDA_ERR_ARG either way round).  Takes effect at
 * the next run; a zda_adjoint needs a zda_forward of the same form. */
zda_status zda_zone_set_radial_pml(zda_zone *zone, int form);
zda_status zda_zone_get_radial_pml(const zda_zone *zone, int *form);

/* Time `steps` time steps of the zone's current step kernel (no source, no
 * DFT) on its current field state, with CUDA events on `stream`; ms_out
 * receives the elapsed milliseconds.  Overwrites the fields (a following
 * zda_adjoint needs a new zda_forward).  Used by the tile-shape tuner. */
zda_status zda_zone_time_steps(zda_zone *zone, int steps, double *ms_out_host, void *stream);

/* The fused and tiled steps (variants 1, 3, 4) wait on shared-memory
 * barriers for their staged copies; every wait gives up after `polls` polls
 * (default 4194304; variants 3 and 4 also after one second), sets an error
 * word and lets the kernel finish, and the call then returns
 * ZDA_ERR_TIMEOUT (zda_forward, zda_adjoint and zda_iteration synchronise
 * their stream to read it).  inject_timeout != 0 is for tests of that path:
 * variant 1 also waits, per radius, on a barrier that nothing completes;
 * variants 3, 4 and 5 once per thread block before their first radius. */
zda_status zda_zone_set_wait_limit(zda_zone *zone, int polls, int inject_timeout);

/* Kernel timing with CUDA events recorded on the launching stream: with
 * every > 0, the main launches of steps every - 1, 2 every - 1, ... are
 * bracketed by events (a ring of 64 samples; the host waits for a sample 64 samples old
 * before reusing its slot).  every = 0 turns it off.
 * zda_zone_timing waits for pending samples and writes ms3_host[0..2], the
 * summed durations (ms) of the step's launches 1, 2, 3 over the sampled
 * steps, and the number of sampled steps, then resets.  Launches 1, 2, 3 are:
 * split step with two z-cells per thread: H update, E update (which also
 * writes the DFT history), DFT flush (only on steps 31, 63, ...: sample
 * with every = 32 to time it);
 * split step with one z-cell per thread: H update, E update (with the DFTs), -;
 * fused step: streaming E/H kernel, -, DFT kernel ("-" reads 0). */
zda_status zda_zone_set_timing(zda_zone *zone, int every);
zda_status zda_zone_timing(zda_zone *zone, double *ms3_host, long long *count_host);

/* Decay probe of forward runs (section "Differentiable FDTD in cylindrical
 * coordinates": the gradient is assembled from the running DFTs of one
 * forward and one adjoint run, which is exact once the time-domain fields
 * have died out by the last step).  With every > 0, each zda_forward (or
 * zda_iteration, or lens forward) records after steps every, 2 every, ...
 *   W    = sum over E sites of eps |E|^2 V + sum over H sites of |H|^2 V,
 *   Wdot = the same sum over the one-step differences (E^{n+1} - E^n and
 *          H^{n+1/2} - H^{n-1/2}),
 * V = r dr dphi dz at the site's radius (E_r, H_phi, H_z at r_{i+1/2}; E_phi,
 * E_z, H_r at r_i), FP64 sums.  Wdot is the decay measure: a source whose
 * time integral is not zero leaves a static charge field that never decays
 * but does not oscillate.  every = 0 (default) turns the probe off.  The
 * split step copies the state before each sampled step into the fused
 * step's second field buffer.  zda_zone_energy_trace copies the samples of
 * the last forward run (n_steps / every of them, at most max_samples) to
 * host arrays and writes their number (synchronous). */
zda_status zda_zone_set_energy_probe(zda_zone *zone, int every);
zda_status zda_zone_energy_trace(zda_zone *zone, double *w_host, double *wdot_host, int max_samples, int *n_samples);

/* Density filter + projection without any device allocation (the paper has
 * no counterpart: this exists for callers that cannot call cudaMalloc, e.g.
 * a program whose device memory belongs to another framework's pool, or a
 * loop that may not allocate once running).  Same result as
 * zda_filter_project, but needs no context, zone or workspace: desc is the
 * zone description (host), rho_dev [n_r_design][n_phi] the density and
 * rho_tilde_dev the output (device, current device), stream a cudaStream_t.
 * Scratch (the filter's per-row weight sums) is a fixed 64 KiB device array
 * inside the library: n_r_design is limited to 16384 rows (ZDA_ERR_ARG
 * beyond).  Accepts what zda_zone_create accepts (wedge zones and the axis
 * zone), including its bound of ZDA_MAX_FILTER_TAPS filter taps per pixel.
 * The first call on each device looks up that array's device address (with
 * that device current) and keeps it; make that first call before any stream
 * capture, and do not use this call on a device after cudaDeviceReset in the
 * same process.  All calls on a device share the array: calls whose kernels
 * overlap on the GPU race.  Allocates nothing. */
zda_status zda_filter_project_noalloc(const zda_zone_desc *desc, const float *rho_dev, float *rho_tilde_dev,
                                      void *stream);

/* ---- lens: all zones of a lens (section "Zoned discrete axisymmetry (ZDA)":
 * concentric zones, each simulated on its own, whose fields add up at the
 * focus).  The caller creates the zones (same wavelengths and focal
 * distance; an axis zone may be first) and binds their workspaces, then the
 * lens and its small workspace.  zda_lens_forward runs every zone's forward
 * solve -- as parallel branches of one CUDA graph replayed per call (captured
 * on first use, and again after a zone's kernel or workspace changes), each
 * zone with its own dt and step count -- and sums the zones' focal phasors on
 * the device: focal_out_host = sum_z S_z (n_freq complex doubles).
 * zda_lens_adjoint gives every zone the same dI/dS (the lens phasor is the
 * plain sum) and writes each zone's dI/drho.  Device buffers: rho_dev[z] and
 * grad_rho_dev[z] are arrays (host) of n_zones device pointers.  Both calls
 * synchronise `stream`.  The lens keeps its own streams and graphs; it owns
 * no device memory beyond what the graph runtime needs. */
zda_status zda_lens_create(zda_ctx *ctx, zda_zone *const *zones, int n_zones, zda_lens **out);
void zda_lens_destroy(zda_lens *lens);
zda_status zda_lens_workspace_bytes(const zda_lens *lens, size_t *bytes);
zda_status zda_lens_bind_workspace(zda_lens *lens, void *workspace_dev, size_t bytes);
zda_status zda_lens_set_graph(zda_lens *lens, int use_graph);     /* 0: enqueue directly, no graph */
zda_status zda_lens_forward(zda_lens *lens, const float *const *rho_dev, double *focal_out_host, void *stream);
zda_status zda_lens_adjoint(zda_lens *lens, const double *dI_dfocal_host, float *const *grad_rho_dev, void *stream);
/* zone z's own phasors S_z from the last zda_lens_forward (host copy). */
zda_status zda_lens_zone_focal(const zda_lens *lens, int zone, double *focal_out_host);
long long zda_lens_launch_count(const zda_lens *lens);   /* graph launches (or direct runs) issued */

/* Focal-plane evaluation after zda_lens_forward (section "Centimeter-scale
 * metalens": focusing efficiency within 3 FWHM, Eq. 9's Strehl ratio with the
 * power transmitted through the whole lens).  pts_dev: n_pts (x, y) doubles
 * in the focal plane (origin on the axis).  field_dev (caller-allocated,
 * 2 * n_lambda * n_pts complex doubles) receives E_x for every wavelength
 * and point, then E_y: Rayleigh-Sommerfeld (first kind) of each zone's
 * azimuthal orders +-1 (its phi-averaged near field), integrated with
 * n_phi_samples (>= 8) azimuthal samples, summed over zones.  p_trans_host
 * (n_lambda doubles, may be NULL): (n/2) |E_t|^2 over all monitor annuli
 * and the whole circle (all azimuthal orders of the wedge; the cross term of
 * the orders +1 and -1 cancels over the n wedge copies for n >= 3 and is
 * kept for n = 1, 2), the transmitted power.  Synchronises `stream`. */
zda_status zda_lens_focal_plane(zda_lens *lens, const double *pts_dev, int n_pts, int n_phi_samples,
                                double *field_dev, double *p_trans_host, void *stream);

/* The same field at points off the focal plane (the far-field maps of
 * "Results and Discussion", e.g. the xz-plane intensity): pts_dev holds
 * n_pts (x, y, h) doubles, h = height above the focal plane (the
 * propagation distance from each monitor plane becomes its focal distance
 * + h).  field_dev as for zda_lens_focal_plane.  Synchronises `stream`. */
zda_status zda_lens_field_points(zda_lens *lens, const double *pts_dev, int n_pts, int n_phi_samples,
                                 double *field_dev, void *stream);

/* Focal-spot evaluation after zda_lens_forward (section "Centimeter-scale
 * metalens at long-wave infrared": the PSF and its full width at half
 * maximum; the absolute focusing efficiency FE = the power inside a disc of
 * radius 3 FWHM around the focus / the incident power on the lens aperture;
 * the relative efficiency = the same / the power transmitted through the
 * lens; Eq. 9's Strehl ratio SR = I(0) lambda^2 F^2 / (P_trans A), A = pi
 * lens_radius^2).  All on the device: the PSF line I(x) = (n_top/2)
 * (abs(E_x)^2 + abs(E_y)^2) at n_line >= 2 points x_i = i x_max /
 * (n_line - 1) on the focal plane's x axis; the FWHM from its first sample
 * below half of I(0) (linear interpolation with the sample before; NaN if
 * none); per wavelength a disc of n_rad radii (k + 1/2) 3 FWHM / n_rad x
 * n_ang angles, its power by the midpoint rule in r and the mean over the
 * angles.  Fields from the lens-field transform of zda_lens_focal_plane with
 * n_phi_samples (>= 8) azimuthal samples; P_trans as there.
 * incident_host: n_lambda incident plane-wave intensities (n/2) abs(E)^2
 * (zda_zone_incident_intensity).  scratch_dev: caller-owned device memory,
 * 256-byte aligned, of at least zda_lens_evaluate_scratch_bytes bytes (the
 * library allocates nothing).  out_host (n_lambda x 8 doubles): per
 * wavelength FWHM, I(0), FE, relative FE, transmittance P_trans / P_inc,
 * SR, disc power, P_trans.  line_dev (optional, n_lambda x n_line doubles,
 * device) receives the PSF line.  At most 8 wavelengths.  Synchronises
 * `stream`. */
zda_status zda_lens_evaluate_scratch_bytes(const zda_lens *lens, int n_line, int n_rad, int n_ang, size_t *bytes);
zda_status zda_lens_evaluate(zda_lens *lens, double lens_radius, double focal, const double *incident_host,
                             double n_top, int n_line, double x_max, int n_rad, int n_ang, int n_phi_samples,
                             void *scratch_dev, size_t scratch_bytes, double *out_host, double *line_dev,
                             void *stream);

/* Incident plane-wave intensity of a reference run: after zda_forward of a
 * zone whose layers and design are all the substrate (no interface, no
 * lens), the phi-mean u of the monitor's E_r phasor over the radii between
 * the r-PMLs, each row's Bloch phase e^{i m phi_j} removed, is half the
 * plane-wave amplitude; out_dev (n_lambda doubles, device) = (n_sub/2)
 * abs(2 u)^2, n_sub = sqrt of the permittivity of the layer at k = 0. */
zda_status zda_zone_incident_intensity(zda_zone *zone, double *out_dev, void *stream);

/* Intensity (n_top/2)(abs(E_x)^2 + abs(E_y)^2) of field samples in the layout
 * of zda_lens_focal_plane / zda_lens_field_points (E_x of every wavelength
 * and point, then E_y; complex doubles): out_dev[l n_pts + p] (device). */
zda_status zda_field_intensity(const double *field_dev, int n_lambda, int n_pts, double n_top, double *out_dev,
                               void *stream);

/* Encircled power of radially symmetric spots: for each of n_prof profiles
 * I_dev[q n + k] sampled at the increasing radii radii_dev[k] (k < n),
 * out_dev[q n + k] = the trapezoid-rule integral of I(r) 2 pi r from
 * radii[0] to radii[k] (device arrays). */
zda_status zda_encircled_power(const double *radii_dev, const double *I_dev, int n_prof, int n, double *out_dev,
                               void *stream);

/* Estimate of what the lens-field transforms above neglect for one zone
 * (host only, no device work).  They keep the azimuthal orders +-1 of the
 * zone's near field; the wedge's other orders m + j n (j != 0) reach a point
 * at distance rho from the axis through Bessel functions J_L(x) with
 * abs(L) >= n - 2 and x <= k r_hi rho / z_f (first order in r rho / R),
 * k = 2 pi n_top / lambda_min, r_hi the zone's outer radius, z_f the point's
 * distance from the monitor plane (focal - monitor height above the design
 * top, + h for (x, y, h) points).  *bound_host = max over the points of
 * (x/2)^nu / Gamma(nu + 1) >= abs(J_nu(x)), nu = max(n - 2, 0): a bound on
 * the neglected orders' kernel relative to the kept one's; 0 for continuous
 * axisymmetry (nothing neglected); HUGE_VAL for a point at or below the
 * monitor plane.  pts_host: n_pts points of `stride` doubles, stride 2
 * (x, y) or 3 (x, y, h). */
zda_status zda_zone_order_bound(const zda_zone_desc *desc, const double *lambda_host, int n_lambda,
                                const double *pts_host, int n_pts, int stride, double *bound_host);

/* Thread-local message of the last error ("" if none). */
const char *zda_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* ZDA_H */
