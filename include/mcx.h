/*
 * mcx.h -- C ABI of the GB300-native forward Monte Carlo X-ray ray tracer.
 *
 * The library traces independent rays (position, direction, energy, Monte
 * Carlo weight) from a source through an ordered list of components, in the
 * model of McXtrace described in arXiv 2410.08747:
 *   - an instrument is a sequential list of components placed relative to
 *     each other (Sec. 2.1, the instrument file and its AT ... RELATIVE
 *     placement);
 *   - rays are generated at the source and propagated through every
 *     component in order; any component may absorb the ray (Sec. 1);
 *   - rays are independent, so the ray ensemble is the unit of parallelism
 *     (Sec. 2.2);
 *   - the particle state holds position, wavevector and weight p (Sec. 2.2.2);
 *     here the wavevector is stored as a unit direction plus the energy E,
 *     |k| = E / (hbar c);
 *   - monitors record count, sum of weights and sum of squared weights per bin
 *     and must be updated race-free by concurrent rays (Sec. 2.2.2);
 *   - all instrument data is copied to the device once and stays resident,
 *     so no host<->device traffic occurs while tracing (Sec. 4.2, where
 *     repeated transfers made the GPU port ~100x slower than expected).
 *
 * Every ray i of a trace under seed s draws its random numbers from
 * Philox4x32-10 (Salmon et al., SC'11) with counter (i mod 2^32, i / 2^32,
 * block, instrument id) and key (s mod 2^32, s / 2^32), so any ray range can
 * be traced anywhere and the sums over sub-ranges equal the sum over the
 * whole range (the scatter/gather of Sec. 2.2.1).
 *
 * Units: metres, keV, 1/m, Angstrom (wavelength).  Frames: a component's
 * local z axis is its optical axis; x_parent = pos + rot * x_local.
 *
 * Threading: calls on one instrument must not overlap; different instruments
 * may be used from different host threads.  Device work is queued on the
 * instrument's stream; calls that return data synchronise that stream.
 *
 * Errors: every call returns an mcx_status.  No call throws, traps or aborts.
 * mcx_last_error() gives a message for the calling thread's last failure.
 */
#ifndef MCX_H
#define MCX_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  MCX_OK = 0,
  MCX_ERR_INVALID = -1,      /* bad argument or instrument description */
  MCX_ERR_OOM = -2,          /* device allocation failed */
  MCX_ERR_CUDA = -3,         /* a CUDA runtime call failed */
  MCX_ERR_TIMEOUT = -4,      /* a bounded device wait gave up */
  MCX_ERR_DEVICE = -5,       /* a kernel reported an error status */
  MCX_ERR_UNSUPPORTED = -6   /* valid request the library does not implement */
} mcx_status;

typedef enum {
  MCX_SOURCE = 0,      /* component 0 only */
  MCX_SLIT_RECT = 1,
  MCX_SLIT_CIRC = 2,
  MCX_ABS_BOX = 3,
  MCX_ABS_CYL = 4,
  MCX_ABS_SPHERE = 5,
  MCX_PHANTOM = 6,
  MCX_MON_PSD = 7,
  MCX_MON_E = 8,
  MCX_MON_L = 9,
  MCX_MON_EPSD = 10,
  MCX_LENS_PARAB = 11  /* compound refractive lens (Sec. 3.2) */
} mcx_comp_type;

typedef enum {
  MCX_SHAPE_POINT = 0, MCX_SHAPE_DISK = 1, MCX_SHAPE_RECT = 2,
  MCX_SHAPE_GAUSS = 3   /* Gaussian spot and divergence (undulator source, Sec. 3.2) */
} mcx_source_shape;
typedef enum { MCX_SPEC_FLAT = 0, MCX_SPEC_KRAMERS = 1, MCX_SPEC_GAUSS = 2 } mcx_spectrum;

typedef enum {
  MCX_PREC_FP64 = 0,   /* plain form: every quantity in binary64 */
  MCX_PREC_MIXED = 1   /* binary32 propagation inside component frames; binary64
                          lab frame, frame transforms and monitor sums */
} mcx_precision;

/*
 * One component.  `p` by type (lengths in m, energies in keV):
 *   SOURCE     shape, spectrum; p0 disk radius or spot width, p1 spot height,
 *              p2 e_min, p3 e_max, p4 Kramers e0 (>= e_max), p5 target
 *              distance D, p6 target width, p7 target height.  Rays start in
 *              the local z = 0 plane, aim at a uniform point of the target
 *              rectangle centred at (0, 0, D), and take E uniform in
 *              [e_min, e_max) with weight 1 (flat) or (e0 - E)/E divided by
 *              its mean over the band (Kramers bremsstrahlung shape).
 *              Gaussian shape (MCX_SHAPE_GAUSS, the undulator source of
 *              Sec. 3.2): p0, p1 standard deviations of x and y, drawn by
 *              Marsaglia's polar method (16 pairs at most, else 0) with a
 *              logarithm built from IEEE operations (x = m 2^e,
 *              f = (m-1)/(m+1), the atanh series to f^20 in binary64, f^10
 *              in binary32); p9, p10 standard deviations of the divergence:
 *              the weight is multiplied by exp(-theta^2 / 2 p9^2) per axis,
 *              theta = (aim - source point) / p5 (0: no weight).
 *              Gaussian spectrum (MCX_SPEC_GAUSS): E = p4 + p8 z, z from a
 *              polar pair drawn after the aim point; e_min, e_max only
 *              bound the mu tables' use.
 *   SLIT_RECT  p0 xmin, p1 xmax, p2 ymin, p3 ymax (closed opening in z = 0)
 *   SLIT_CIRC  p0 radius
 *   ABS_BOX    p0..p2 full widths wx, wy, wz; material
 *   ABS_CYL    p0 radius, p1 height (axis = local y); material
 *   ABS_SPHERE p0 radius; material
 *   PHANTOM    p0 voxel edge; n = (nx, ny, nz); bytes from mcx_phantom;
 *              p1 = s in [0, 64]: 0 integrates mu exactly along the line
 *              (voxel-boundary walk); s > 0 takes the fixed-step traversal
 *              of Sec. 3.3 instead: steps of p0 / s from the grid entry,
 *              each weighted by the voxel holding its end point (clamped),
 *              the last one cut at the grid exit, positions in 32.32
 *              fixed-point voxel coordinates rounded once from binary64
 *              (p2, p3 are overwritten by the library).  p4 != 0 (with
 *              s > 0 and mcx_phantom.mu_scatter): each step may also
 *              scatter the ray (Sec. 3.3): the scattering depth of the
 *              steps is added up
 *              in the decision type, and when it reaches -ln(1 - u) (a
 *              draw at the grid entry and after each scattering, the
 *              contract's logarithm) the ray scatters at the step's end
 *              point and is marched on from there (at most 8
 *              scatterings).  The scattering depth of a step is
 *              (mu_R(E) + mu_C(E)) len of its voxel's material, each
 *              coefficient from its table at the ray's energy in the
 *              decision type (looked up again, with the attenuation
 *              ahead, after a Compton event); the event is
 *              Compton when a draw falls below mu_C / (mu_R + mu_C), else
 *              Rayleigh; its polar angle by rejection against the Thomson
 *              law 1 + mu^2 or the Klein-Nishina law (16 pairs at most,
 *              else forward), Compton lowering E to E / (1 + (E/m_e c^2)
 *              (1 - mu)); its azimuth from a point of the unit disc.  A scattered
 *              ray leaves the phantom from its exit point on its new line.
 *              Instruments with a scattering phantom cannot trace given
 *              starts (the draws continue the ray's own stream).
 *   MON_PSD    p0..p3 xmin, xmax, ymin, ymax; n = (nx, ny, -)
 *   MON_E      p0..p3 aperture; p4 e_min, p5 e_max; n0 = bins
 *   MON_L      p0..p3 aperture; p4 l_min, p5 l_max (Angstrom); n0 = bins
 *   MON_EPSD   p0..p3 extent; p4 e_min, p5 e_max; n = (nx, ny, ne);
 *              bin index = (iy * nx + ix) * ne + ie
 *   LENS_PARAB compound refractive lens (Sec. 3.2): n0 = N double-sided
 *              parabolic lenses centred on the origin, lens j at
 *              z_j = (j - (N-1)/2) p6; its surfaces z = z_j -/+ (p1/2 +
 *              (x^2 + y^2) / (2 p0)) (p0 apex radius of curvature, p1 apex
 *              thickness), aperture radius p2 (a ray outside it at a surface
 *              is absorbed); refractive index 1 - delta with
 *              delta = p4 (p5 / E)^2; p3 = N as a real.  Each surface is
 *              met by the cancellation-free root of its quadratic and
 *              refracted by the vector Snell law written with eta - 1 and
 *              eta^2 - 1 formed from delta; the path between the surfaces
 *              attenuates the weight by exp(-mu_material(E) L).  The ray
 *              leaves with its new position and direction.
 *   MON_*      p11 restore: when nonzero the ray leaves the monitor as it
 *              entered it (its position is not moved to the monitor plane),
 *              and a ray that cannot reach the plane passes unscored instead
 *              of being absorbed.  Several tilted monitors around one beam
 *              (the five line detectors of the paper's EDXCT instrument,
 *              Sec. 3.3) each see every ray this way, whatever their order.
 * Absorbers keep the ray's line and multiply its weight by exp(-mu(E) L),
 * L the chord of the half-line in the solid.  Planar components (slits and
 * monitors) first move the ray to their z = 0 plane and absorb it if it
 * cannot get there (k_z = 0 or a negative path), restoring monitors
 * excepted.  Monitors never absorb otherwise; bins are half-open and
 * out-of-range values are not counted.
 */
typedef struct {
  int32_t type;          /* mcx_comp_type */
  int32_t relative_to;   /* -1: lab frame; else index of an earlier component */
  int32_t shape;         /* mcx_source_shape (SOURCE) */
  int32_t spectrum;      /* mcx_spectrum (SOURCE) */
  int32_t material;      /* material index (absorbers) */
  int32_t n[3];          /* bin or voxel counts */
  double pos[3];         /* origin in the parent frame */
  double rot[9];         /* row-major rotation local -> parent */
  double p[12];          /* type parameters, see above */
} mcx_component_desc;

/* Attenuation tables: on cell j of [e_min, e_max) split into n_cell equal
 * cells, mu_m(E) = coef[(m * n_cell + j) * 2] + coef[(m * n_cell + j) * 2 + 1] * E
 * in 1/m, j = floor((E - e_min) * n_cell / (e_max - e_min)) clamped to the
 * table.  Host memory owned by the caller; copied at create. */
typedef struct {
  int32_t n_mat;
  int32_t n_cell;
  double e_min, e_max;
  const double* coef;
} mcx_material_tables;

/* Voxel phantom: nx*ny*nz material bytes, x fastest ([nz][ny][nx]), each
 * < n_mat.  Host memory owned by the caller; copied at create. */
typedef struct {
  const uint8_t* vox;
  int32_t nx, ny, nz;
  /* Scattering phantom (PHANTOM p4 != 0, on the fixed-step march p1 > 0,
   * at most 32 materials): the Rayleigh (elastic) scattering coefficient
   * table, [n_mat][n_cell][2] in the layout of mcx_material_tables.coef
   * (mu = c0 + c1 E on each cell, 1/m; an energy-independent coefficient
   * is c1 = 0), and optionally (NULL: none) the Compton table of the same
   * shape.  Each line must be finite and >= 0 on its cell (the first cell
   * from E = 0), else MCX_ERR_INVALID.  Host memory owned by the caller;
   * copied at create. */
  const double* mu_scatter;
  const double* mu_compton;
} mcx_phantom;

/* Device allocation hook: when `alloc` is non-NULL every device buffer of the
 * instrument comes from alloc(bytes, ctx) (256-byte aligned, device memory of
 * `device`) and goes back through free(ptr, ctx); otherwise cudaMalloc. */
typedef struct {
  int32_t precision;     /* mcx_precision */
  int32_t instr_id;      /* Philox counter word 3; < 2^31 */
  int32_t device;        /* CUDA device ordinal */
  int32_t block_size;    /* threads per block, 0 = library default */
  int32_t blocks_per_sm; /* resident blocks per SM, 0 = library default */
  int32_t reserved;
  void* (*alloc)(size_t bytes, void* ctx);
  void (*free)(void* ptr, void* ctx);
  void* alloc_ctx;
  void* stream;          /* cudaStream_t; NULL = legacy default stream */
} mcx_options;

typedef struct mcx_instrument mcx_instrument;

/* Validate, place and upload an instrument.  `mats` may be NULL when no
 * component needs a material; `ph` may be NULL without a PHANTOM.  All
 * inputs are copied; monitors start at zero.  On success *out owns device
 * memory until mcx_instrument_destroy. */
mcx_status mcx_instrument_create(const mcx_component_desc* comps, int32_t n_comps,
                                 const mcx_material_tables* mats, const mcx_phantom* ph,
                                 const mcx_options* opt, mcx_instrument** out);

/* Trace rays [ray_begin, ray_end) under `seed`, adding to the monitors and
 * tallies (stream-ordered, returns before the device finishes).  Tracing a
 * range twice counts it twice. */
mcx_status mcx_trace_range(mcx_instrument* inst, uint64_t ray_begin, uint64_t ray_end,
                           uint64_t seed);

/* mcx_trace_range(inst, 0, n_rays, seed). */
mcx_status mcx_trace(mcx_instrument* inst, uint64_t n_rays, uint64_t seed);

/* Instrument compilation (McXtrace compiles each instrument description to
 * its own program, arXiv 2410.08747 Sec. 2.1).  enable != 0: generate a
 * tracing kernel whose component table (types, placed frames, parameters)
 * is a compile-time constant, compile it for this GPU at run time (NVRTC,
 * --fmad=false, the same arithmetic as the generic kernel) and use it for
 * every later mcx_trace / mcx_trace_range of `inst`; identical instruments
 * share one compiled kernel per process.  enable == 0: back to the generic
 * kernel.  Synchronous; the first compilation of a table takes seconds.
 * MCX_ERR_UNSUPPORTED when the run-time compiler is unavailable or fails (the
 * generic kernel stays in use), or a parameter is not finite. */
mcx_status mcx_instrument_specialize(mcx_instrument* inst, int32_t enable);

/* The source text of inst's specialised kernel, NUL-terminated.  *len (if
 * not NULL) receives the size including the NUL; with buf != NULL, cap must
 * be at least that size.  Pure host call. */
mcx_status mcx_instrument_source(const mcx_instrument* inst, char* buf, size_t cap, size_t* len);

/* Number of bins of monitor component `comp_index`. */
mcx_status mcx_monitor_bins(const mcx_instrument* inst, int32_t comp_index, size_t* n_bins);

/* Copy monitor `comp_index` into caller-owned host arrays of exactly n_bins
 * entries (any of the three may be NULL).  When every given array is
 * page-locked host memory the device can address (cudaHostAlloc under
 * unified addressing), one kernel splits the bins straight into them over
 * the host link.  Otherwise the bins are split on the device into a scratch
 * of 24 bytes per bin of the largest monitor, which the first such read
 * allocates (through the instrument's allocator) and destroy frees, and the
 * host arrays receive plain copies.  Synchronises the stream.
 * MCX_ERR_OOM when the scratch cannot be allocated. */
mcx_status mcx_monitor_read(mcx_instrument* inst, int32_t comp_index, uint64_t* N,
                            double* sum_w, double* sum_w2, size_t n_bins);

/* The read of mcx_monitor_read queued on the instrument's stream without
 * waiting for it (Sec. 2.2.2's monitors, as they stand when the stream
 * reaches the read): the bins are split on the device into the readout
 * scratch (allocated by the first read, as above), then three DMA copies
 * bring them into the caller's host arrays (n_bins entries each, any may be
 * NULL).  With page-locked arrays the copies run on the copy engines, so a
 * readout can overlap a trace queued on another instrument's stream; the
 * arrays may be read, and must stay alive and untouched, only after
 * mcx_synchronize(inst) (or any later synchronising call on the instrument)
 * has returned.  The next read or trace of the same instrument is ordered
 * after this one by its stream.  Pageable arrays work too, but each copy
 * into pageable memory waits for the device.  MCX_ERR_OOM when the scratch
 * cannot be allocated. */
mcx_status mcx_monitor_read_async(mcx_instrument* inst, int32_t comp_index, uint64_t* N,
                                  double* sum_w, double* sum_w2, size_t n_bins);

/* Totals over the bins of monitor `comp_index`: the count, the sum of
 * weights and the sum of squared weights of every ray it scored (the
 * detector-integrated tally; the intensity estimate is sum_w / rays
 * emitted, Sec. 2.2.2), reduced on the device (count exact, sums in
 * binary64 in no fixed order) into caller-owned host scalars (any may be
 * NULL).  The first call allocates 32 bytes through the instrument's
 * allocator.  Synchronises the stream. */
mcx_status mcx_monitor_total(mcx_instrument* inst, int32_t comp_index, uint64_t* N, double* sum_w,
                             double* sum_w2);

/* Copy the tallies: per component the weight it removed (absorbed rays, or
 * w (1 - exp(-tau)) at absorbers), n entries (n = component count); rays
 * emitted; total emitted weight; weight still alive after the last
 * component.  Any pointer may be NULL.  Synchronises the stream. */
mcx_status mcx_tally_read(mcx_instrument* inst, double* lost, int32_t n, uint64_t* n_emit,
                          double* sum_w0, double* sum_wend);

/* The per-component loss tally alone (the weight each component removed:
 * absorbed rays, or w (1 - exp(-tau)) at absorbers; paper Sec. 2.2.2, a
 * component may absorb the ray), n entries (n = component count), in
 * caller-owned host memory: mcx_tally_read with only `lost`.  Synchronises
 * the stream. */
mcx_status mcx_loss_read(mcx_instrument* inst, double* per_component_lost_w, int32_t n);

/* Zero every monitor and tally (stream-ordered). */
mcx_status mcx_monitor_reset(mcx_instrument* inst);

/* Wait for the instrument's queued work and report any deferred error. */
mcx_status mcx_synchronize(mcx_instrument* inst);

/* Release the instrument and its device memory (NULL is ignored). */
void mcx_instrument_destroy(mcx_instrument* inst);

/* Message of the calling thread's last failed call ("" if none). */
const char* mcx_last_error(void);

/* ---------------------------------------------------------------- ray starts
 * A ray start is what the source draws for a ray before propagation: source
 * point (sx, sy) in the source frame, aim point (u, v) on the target plane,
 * energy E, and initial weight w0.  A start buffer is a DEVICE array of 6 n
 * floats laid out as rows sx[n], sy[n], E[n], u[n], v[n], w0[n].  Separating
 * the two steps lets a different sampler (the learned proposal below) feed
 * the same tracer, and lets the tracer report per-ray detector outcomes, the
 * ray histories the proposal is trained on. */

/* Write the starts of rays [ray_begin, ray_begin + n) as the instrument's own
 * source samples them (binary32 draws, Kramers weight) into d_starts
 * (caller-owned device memory).  Stream-ordered. */
mcx_status mcx_sample_starts(mcx_instrument* inst, uint64_t ray_begin, uint64_t n, uint64_t seed,
                             float* d_starts);

/* Trace n rays from the given starts (ray ids ray_base..; mixed precision
 * only), adding to the monitors and tallies.  d_det_w (device, n floats, may
 * be NULL) receives each ray's weight as scored by the last component when
 * that is a monitor (0 if the ray is not scored there).  A start with w0 = 0
 * counts as emitted but is not traced.  Tracing starts from mcx_sample_starts
 * equals mcx_trace_range on the same rays.  Stream-ordered. */
mcx_status mcx_trace_starts(mcx_instrument* inst, const float* d_starts, uint64_t n,
                            uint64_t ray_base, float* d_det_w);

/* ---------------------------------------------------------------- learned proposal
 * An importance-sampling density for a source's aim point, learned from ray
 * histories.  The paper motivates it without defining it: most simulated
 * rays are wasted (stopped by a slit or missing the detector, Sec. 3.2) and
 * an energy-dispersive CT projection needs >= 1e7 rays (Sec. 5.1).
 *
 * Network: x -> 3 hidden layers of 128 SiLU units -> 40 outputs, y = x W + b,
 * with x_i = (raw_i - x_shift[i]) x_scale[i] and raw = (source x, source y,
 * energy, projection angle).  Outputs per component k = 0..7: (logit, mu_u,
 * mu_v, r_u, r_v); pi = softmax(logits), log sigma = 2.5 tanh(r / 2.5) - 2.5,
 * a Gaussian mixture over the normalised aim point (u / half_u, v / half_v).
 * Parameters: 38824 floats, in the order W1 [4,128], b1, W2 [128,128], b2,
 * W3 [128,128], b3, W4 [128,40], b4 (row-major [in, out]).  Hidden and output
 * layers run on BF16 tensor cores with FP32 accumulation; the master copy is
 * FP32.
 *
 * Sampling draws the aim point from alpha U(window) + (1 - alpha) mixture;
 * an aim point outside the window gets weight 0, otherwise the start's weight
 * is the source's Kramers weight times (1/4) / q (the plain sampler is
 * uniform on the window), so the estimator stays unbiased for alpha > 0. */
typedef struct mcx_proposal mcx_proposal;

typedef struct {
  float alpha;            /* defensive uniform fraction, (0, 1] */
  float half_u, half_v;   /* half sizes of the aim window (m) */
  float x_shift[4];       /* input normalisation */
  float x_scale[4];
  int32_t device;
  int32_t reserved;
  void* stream;           /* cudaStream_t for training and diagnostics */
} mcx_proposal_desc;

typedef struct {
  uint32_t epochs;        /* passes over the history */
  uint32_t batch;         /* rows per Adam step, in [128, 2^20] */
  float lr, beta1, beta2, eps;
} mcx_train_opts;

/* Create a proposal; params (host, 38824 floats) may be NULL for zeros. */
mcx_status mcx_proposal_create(const mcx_proposal_desc* desc, const float* params,
                               mcx_proposal** out);
/* Copy parameters in (resets the Adam state) or out; host arrays of 38824. */
mcx_status mcx_proposal_set_params(mcx_proposal* p, const float* params);
mcx_status mcx_proposal_get_params(mcx_proposal* p, float* params);

/* Diagnostics on device rows: network outputs (d_out: n x 40 floats) for
 * normalised inputs d_x (n x 4); and the weighted NLL of targets d_t (n x 2,
 * normalised aim points) with weights d_w (n), plus its gradient (host, 38824
 * floats).  n <= 2^24.  Synchronise the proposal's stream. */
mcx_status mcx_proposal_forward(mcx_proposal* p, const float* d_x, uint64_t n, float* d_out);
mcx_status mcx_proposal_loss_grad(mcx_proposal* p, const float* d_x, const float* d_t,
                                  const float* d_w, uint64_t n, double* loss, float* grad);

/* Train on a ray history: d_starts (n starts, mcx_sample_starts layout) and
 * d_det (n detected weights from mcx_trace_starts), all rows with the given
 * projection angle; Adam on mini-batches of opt->batch consecutive rows
 * (a trailing partial batch is skipped).  *last_loss receives the last
 * batch's loss.  Synchronises. */
mcx_status mcx_proposal_train(mcx_proposal* p, const float* d_starts, const float* d_det, uint64_t n,
                              float angle, const mcx_train_opts* opt, double* last_loss);

/* mcx_proposal_train with a projection angle per row: d_angle (device, n
 * floats) gives row i's angle input, so that a history gathered over many
 * projections of a scan (rows shuffled across angles) trains one network
 * for all of them, every mini-batch mixing angles. */
mcx_status mcx_proposal_train_angles(mcx_proposal* p, const float* d_starts, const float* d_det,
                                     const float* d_angle, uint64_t n, const mcx_train_opts* opt,
                                     double* last_loss);

/* Draw the starts of rays [ray_begin, ray_begin + n) of `inst` (mixed form)
 * from the proposal into d_starts (device, 6 n floats); trace them with
 * mcx_trace_starts.  One persistent kernel: the network runs on the tensor
 * cores (tcgen05, accumulators in tensor memory), 128 rays per warpgroup.
 * Stream-ordered on the instrument's stream; it first waits for that stream
 * to reach this call.  MCX_ERR_TIMEOUT when an earlier call's kernel gave up
 * waiting for the tensor cores (its starts are then incomplete). */
mcx_status mcx_proposal_sample(mcx_proposal* p, mcx_instrument* inst, uint64_t ray_begin, uint64_t n,
                               uint64_t seed, float angle, float* d_starts);

/* Attach proposal p to instrument inst (mixed form, no scattering phantom):
 * from now on mcx_trace and mcx_trace_range of inst draw every ray's start
 * from p at projection angle `angle` instead of the source's own sampler:
 * the rays are sampled and traced 2^23 at a time through a start buffer of
 * the instrument (200 MB, allocated by the first attach through the
 * instrument's allocator, kept until destroy).  Results equal
 * mcx_proposal_sample followed by
 * mcx_trace_starts over the same rays.  p = NULL detaches (the source
 * samples again).  p must outlive the attachment.  mcx_batch_trace draws
 * an attached instrument's starts from p too (see there); the
 * allocation-free mcx_batch_trace_static refuses such instruments
 * (MCX_ERR_UNSUPPORTED).  Each later trace call first
 * reads p's tensor-core status (synchronising the stream) and returns
 * MCX_ERR_TIMEOUT if an earlier sample of p gave up. */
mcx_status mcx_proposal_attach(mcx_instrument* inst, mcx_proposal* p, float angle);

/* Testing: every tensor-core wait of p's kernels (sampler, forward,
 * gradient) gives up after `polls` polls of its mbarrier (polls < 0: the
 * default, 2^24; 0: at once), sets p's timeout status and frees its tensor
 * memory after draining the operations in flight with the default limit.  A
 * later call on p then returns MCX_ERR_TIMEOUT (the status stays set for the
 * proposal's lifetime); other proposals and instruments are unaffected.
 * Lets a test make the bounded wait run out without any device fault. */
mcx_status mcx_proposal_set_wait_limit(mcx_proposal* p, int64_t polls);

void mcx_proposal_destroy(mcx_proposal* p);

/* ---------------------------------------------------------------- batches
 * Many instruments with uneven ray budgets traced by one persistent launch:
 * the budgets are cut into work items of `chunk_rays` consecutive ray ids,
 * ordered by instrument, and resident blocks take items from a device ticket
 * counter until none is left (no block ever waits on another).  An
 * instrument whose monitors in global memory exceed 16 MB gets shorter items
 * (c rays, c the largest power of two with grid x c <= budget, at least
 * 4096 and at most chunk_rays), so that the items in flight at once score
 * into about one detector that the L2 can hold.  Results equal
 * tracing each instrument alone over [0, budget) under the same seed: ray
 * streams are counter-based (Sec. 2.2, independent rays; Sec. 2.2.1, work
 * split over workers and summed).  A CT scan, many projections of one
 * instrument, is the motivating case (Sec. 3.3, Sec. 5.1). */
typedef struct mcx_batch mcx_batch;

typedef struct {
  uint64_t chunk_rays;   /* rays per work item; 0 = 1 << 20 */
  int32_t block_size;    /* threads per block (multiple of 32, <= 256); 0 = 256 */
  int32_t blocks_per_sm; /* resident blocks per SM; 0 = occupancy limit */
  int32_t use_graph;     /* nonzero: capture the launch in a CUDA graph, replay it */
  int32_t reserved;
} mcx_batch_options;

/* `insts` (n >= 1, not owned) must share device, precision and stream and
 * stay alive until mcx_batch_destroy; budgets[i] is the ray count of insts[i]
 * (ray ids [0, budgets[i])).  opt may be NULL (defaults). */
mcx_status mcx_batch_create(mcx_instrument* const* insts, const uint64_t* budgets, int32_t n,
                            const mcx_batch_options* opt, mcx_batch** out);

/* Trace every instrument of the batch under `seed`, adding to each one's
 * monitors and tallies (stream-ordered).  Staged instruments, those with a
 * proposal attached (mcx_proposal_attach, which then draws their starts as
 * mcx_trace would) and, in the mixed form, those with a phantom that does
 * not scatter, go in waves of at most 2^23 rays: each wave's starts are
 * sampled into a buffer of the batch (200 MB, allocated by the first such
 * trace, with 300 MB more behind a phantom), a phantom's put in aim-tile
 * order (the ray order of a single instrument's phantom trace; given starts
 * carry all of a ray's randomness, so the order changes only the order of
 * the atomic additions), then one persistent launch traces the wave, the
 * first wave also carrying every other instrument's budget.  Results equal
 * tracing each instrument alone.  A batch with staged instruments launches
 * directly, without the graph, and first reads each attached proposal's
 * tensor-core status (synchronising the stream; MCX_ERR_TIMEOUT if an
 * earlier sample gave up). */
mcx_status mcx_batch_trace(mcx_batch* b, uint64_t seed);

/* Try launch shapes (block size, resident blocks, chunk size) on a sample of
 * at most `sample_rays` rays per instrument (each shape timed twice), keep
 * the one with the smallest chunk among those within 5 % of the fastest
 * (a sample cannot show what chunk size does at full size: on a batch of
 * 376 instruments with 100 MB detectors, 2^16-ray chunks ran 1.45x faster
 * than 2^18 ones that had won the sample by a hair) for this batch and
 * cache it per batch shape.  Traces into the instruments' monitors and
 * then resets every monitor and tally of the batch.  `chosen` (may be NULL)
 * receives the kept shape.  Synchronises the stream. */
mcx_status mcx_batch_autotune(mcx_batch* b, uint64_t sample_rays, uint64_t seed,
                              mcx_batch_options* chosen);

/* Compile the batch's tracing kernel by instrument families (enable != 0),
 * or go back to the generic kernel (enable == 0).  McXtrace compiles each
 * instrument description into its own program (arXiv 2410.08747 Sec. 2.1);
 * a batch of many instruments is compiled by families instead: instruments
 * with the same sequence of component types form a family, the component
 * fields every member shares become compile-time constants of the kernel,
 * and the fields that differ (a rotation, a slit's edges) are read from each
 * instrument's table.  All families go into one persistent kernel, which
 * picks an instrument's family per work item, so the batch stays one
 * (graph-captured) launch.  Per-ray results are those of the generic kernel.
 * Compiled with NVRTC at run time (~0.3 s per family; identical batches reuse
 * the kernel).  MCX_ERR_UNSUPPORTED: more than 8 families, a non-finite
 * parameter, or a compiler failure (the batch keeps its current kernel).
 * Resets the captured graph; the next mcx_batch_trace captures again. */
mcx_status mcx_batch_specialize(mcx_batch* b, int32_t enable);

/* Work items of the batch's current plan (for tests and planning). */
mcx_status mcx_batch_items(const mcx_batch* b, uint64_t* n_items);

/* Release the batch (not its instruments); NULL is ignored. */
void mcx_batch_destroy(mcx_batch* b);

/* Batched trace that allocates nothing.  The paper has no counterpart; this
 * call exists for callers that cannot allocate device memory: code whose
 * device memory is owned by another allocator or capped in advance, and code
 * that must not call cudaMalloc/cudaFree because cudaFree synchronises the
 * whole device and both stall other work (such callers create their
 * instruments with the mcx_options allocation hook, then trace here).
 *
 * Traces insts[i] over rays [0, budgets[i]) under `seed`, exactly as
 * mcx_batch_trace would (same monitors and tallies), with work items of
 * `chunk_rays` rays (0 = 1 << 20).  Instead of buffers of its own it uses one
 * fixed scratch array compiled into the library (~52 KB, held by every device
 * that loads the library until the process exits), so n is at most 512 and
 * larger requests fail with MCX_ERR_INVALID.  No cudaMalloc, cudaFree or other
 * allocating routine is called.  The first call on a device looks up the
 * array's device address (cudaGetSymbolAddress).  Every call shares the
 * array and leaves its contents
 * behind (the ticket counter is cleared at the start of each call), so calls
 * whose GPU work overlaps on one device (for example on two streams) race on
 * it: issue them on one stream.  Stream-ordered; returns before the device
 * finishes. */
mcx_status mcx_batch_trace_static(mcx_instrument* const* insts, const uint64_t* budgets, int32_t n,
                                  uint64_t chunk_rays, uint64_t seed);

/* Diagnostic: evaluate the device Philox4x32-10 block function (Salmon et
 * al., SC'11; the generator every ray draws from) on `n` host-supplied inputs
 * ctr_key[6 i .. 6 i + 5] = (c0, c1, c2, c3, k0, k1), writing out[4 i .. 4 i + 3].
 * Host arrays owned by the caller; runs on `device` and synchronises. */
mcx_status mcx_philox_fill(const uint32_t* ctr_key, uint32_t* out, size_t n, int32_t device);

/* Diagnostic: the device's binary64 -> binary32 rounding (to nearest, ties to
 * even) and exact binary32 -> binary64 widening used by the mixed form's frame
 * changes: out_f[i] = round(in[i]), out_d[i] = widen(out_f[i]).  Host arrays
 * of n entries owned by the caller; runs on `device` and synchronises. */
mcx_status mcx_convert_fill(const double* in, float* out_f, double* out_d, size_t n,
                            int32_t device);

/* ---------------------------------------------------------------- peaks
 * Diagnostic: the library's own microbenchmarks of the hardware units the
 * tracer's roofline divides by (the tracer is not a dense contraction; the
 * paper reports speed-ups only, Sec. 4, so these denominators are measured
 * here).  Each kind launches a persistent grid (8 blocks of 256 threads per
 * SM) on a private stream, times six launches with CUDA events and reports
 * the fastest of the last five, in *ops_per_s:
 *   FFMA      binary32 fused multiply-adds per second (lane instructions);
 *   IMAD      32-bit integer multiply-adds per second;
 *   PHILOX    Philox4x32-10 blocks per second (the per-ray generator);
 *   DFMA      binary64 fused multiply-adds per second;
 *   HIT       monitor hits per second: three global atomic adds (u64 count,
 *             f64 sum w, f64 sum w^2) to one 24-byte bin at a uniformly
 *             random bin of an array of footprint_bytes, issued as the
 *             tracer issues them (with its L2 evict-last hint);
 *   RED_U64   u64 global atomic adds per second at random positions of an
 *             array of footprint_bytes.
 * footprint_bytes is used by HIT and RED_U64 only (64 .. 2^32 - 1 elements);
 * those two allocate and free it (cudaMalloc).  Changes no clock or other
 * device setting; synchronises its own stream.  MCX_ERR_INVALID for an
 * unknown kind or footprint. */
typedef enum {
  MCX_PEAK_FFMA = 0, MCX_PEAK_IMAD = 1, MCX_PEAK_PHILOX = 2, MCX_PEAK_DFMA = 3,
  MCX_PEAK_HIT = 4, MCX_PEAK_RED_U64 = 5
} mcx_peak_kind;
mcx_status mcx_peak_measure(int32_t kind, int32_t device, uint64_t footprint_bytes, double* ops_per_s);

#ifdef __cplusplus
}
#endif
#endif
