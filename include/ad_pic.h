/*
 * ad_pic.h - C ABI of the GB300 dual-number 3D space-charge PIC library.
 *
 * The method (Qiang, Hao, Qiang, Wan, "A multi-language auto-differentiation
 * module and its application to a parallel particle-in-cell code on
 * distributed computers"):
 *   - every particle coordinate, grid density, potential and field value is a
 *     first-order dual number (value plus P derivatives), Sec. 2, Eqs. 1-4, and
 *     Sec. 4 ("D r_i, D p_i", "D rho, D phi");
 *   - one step is the split map M1(tau/2) M2(tau) M1(tau/2), Sec. 4, Eq. "map";
 *   - M1 is the drift / thick-quadrupole map with dual k and dual tau, Sec. 4,
 *     Eq. "quadtr" and its dual form; M2 is the space-charge kick, Sec. 4,
 *     Eqs. for r(tau), p(tau);
 *   - the Poisson equation is solved for the value and every derivative
 *     channel (Sec. 4); here in 3D with open boundaries by a Hockney FFT
 *     convolution with an integrated Green's function (the paper's 2D pipe
 *     solver is not this path);
 *   - each period ends with the dual emittance D eps = sqrt(D<x^2> D<px^2> -
 *     (D<x px>)^2), Sec. 4.
 *
 * Conventions for every entry point:
 *   - return 0 on success or a negative AD_PIC_ERR_* status; a failed call
 *     leaves the handle destroyable; ad_pic_strerror() names the status;
 *   - all pointers are HOST pointers unless a name ends in "_dev"; the caller
 *     owns every buffer it passes, the library owns all device memory it
 *     allocates and frees it in ad_pic_destroy();
 *   - a handle is not thread-safe; it launches on one CUDA stream (its own,
 *     or the one given to ad_pic_set_stream) and every call that returns
 *     results synchronizes that stream before returning;
 *   - coordinates are (x, px, y, py, z, delta): positions in m (lab frame,
 *     z relative to the reference particle), momenta normalised by p0
 *     (Sec. 4), delta = dp/p0;
 *   - the particle state layout is [6][N][C] doubles, C = n_deriv + 1,
 *     channel 0 the value and channel k the derivative w.r.t. parameter k.
 */
#ifndef AD_PIC_H
#define AD_PIC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    AD_PIC_OK = 0,
    AD_PIC_ERR_INVALID_ARG = -1, /* a size, pointer or enum is out of range */
    AD_PIC_ERR_OOM = -2,         /* a device or host allocation failed */
    AD_PIC_ERR_CUDA = -3,        /* a CUDA runtime call failed */
    AD_PIC_ERR_STATE = -4,       /* call out of order (e.g. run before set_beam) */
    AD_PIC_ERR_NONFINITE = -5,   /* a particle coordinate became NaN or Inf */
    AD_PIC_ERR_OUT_OF_GRID = -6, /* a particle fell outside the grid stencil */
    AD_PIC_ERR_TIMEOUT = -7,     /* a bounded device wait gave up */
    AD_PIC_ERR_UNSUPPORTED = -8, /* valid request the library does not implement */
    AD_PIC_ERR_IO = -9,          /* a checkpoint file could not be read or written */
    AD_PIC_ERR_UNSTABLE = -10    /* a cell has no periodic Twiss solution (|cos mu| >= 1) */
};

enum { AD_PIC_FP64 = 0, AD_PIC_FP32_MIXED = 1 };

typedef struct ad_pic ad_pic; /* opaque handle */

/* Grid nodes per dimension: powers of two in [8, 128]. */
typedef struct {
    int nx, ny, nz;
} ad_pic_grid;

/* The FODO period of Sec. 1 / Sec. 4: drift D1, focusing quad QF, drift D2,
   defocusing quad QD, drift D3. deriv_slot[j] is the derivative slot
   (0 .. n_deriv-1) of parameter j in the order (L_D1, L_QF, g_QF, L_D2, L_QD,
   g_QD, L_D3) - the order of Sec. 3 and Sec. 4 - or -1 to hold it constant.
   Derivatives are w.r.t. the gradient g in T/m; the normalised strength of
   Sec. 4 is k = q g / p0 = g / (B rho). */
typedef struct {
    double L[5];       /* element lengths (m), > 0 */
    double g[2];       /* QF, QD gradients (T/m), nonzero */
    int kicks[5];      /* space-charge kicks per element, >= 1 */
    int deriv_slot[7];
} ad_pic_lattice;

/* Reference particle and initial distribution. Per plane (x, y, z) the
   initial particles are u = sqrt(eps beta) n1, p = sqrt(eps/beta) (n2 - alpha n1)
   with eps = eps_n / (beta0 gamma0), then the sample mean is removed
   (Sec. 4: initial distribution parameters may be AD variables).
   twiss_deriv_slot gives the slots of (alpha_x, beta_x, eps_x, alpha_y,
   beta_y, eps_y), eps the geometric rms emittance, or -1.
   charge_deriv_slot is the slot of the bunch charge (Sec. 4: the beam
   current as an AD variable) or -1: the macroparticle charge Q / N is then a
   dual number in the deposit, so every field and kick carries d/dQ.
   energy_deriv_slot is the slot of the kinetic energy (Sec. 4: beam
   parameters as AD variables) or -1: gamma0, beta0 gamma0, B rho and the
   kick constants are then duals of the energy, and so is the rest-frame z
   spacing gamma0 hz, which enters the Green's function (one more convolution
   per kick: dG/dE of channel 0 into the energy channel) and E_z. It must
   differ from charge_deriv_slot. Only ad_pic_set_beam accepts it; the batched
   runtime and the 2D pipe return AD_PIC_ERR_UNSUPPORTED for it. */
typedef struct {
    double kinetic_eV, mass_eV, charge_e, bunch_charge_C;
    double eps_n[3];   /* normalised rms emittances (m rad), > 0 */
    double alpha[3];
    double beta[3];    /* m, > 0 */
    int twiss_deriv_slot[6];
    int charge_deriv_slot;
    int energy_deriv_slot;
} ad_pic_beam;

/* Create a handle for n_particles in [1, 2^31 - 1] macroparticles (particle
   indices and cell offsets are 32-bit) on the given grid (nx, ny, nz powers
   of two in [8, 128]) with n_deriv in {7, 13} derivative slots and precision AD_PIC_FP64 (every step
   in FP64) or AD_PIC_FP32_MIXED (particles, deposit, FFT, field and push in
   FP32; grid geometry, Green's-function integrals and all moment reductions
   in FP64). Allocates every device buffer; *out is NULL on failure.
   AD_PIC_ERR_INVALID_ARG for sizes outside these ranges. */
int ad_pic_create(const ad_pic_grid* grid, int64_t n_particles, int n_deriv, int precision, ad_pic** out);

/* Set the reference particle and bunch charge. If normals is not NULL it is
   [6][N] standard-normal draws (n1,n2 per plane x, y, z) and the initial
   dual particles are generated on the device from them; if NULL only the
   physics constants are set and particles must come from ad_pic_set_particles. */
int ad_pic_set_beam(ad_pic* h, const ad_pic_beam* beam, const double* normals);

/* Upload / download the dual particle state [6][N][C] (FP64 on the host,
   rounded to the handle's precision on upload). Resets the kick counter
   only in ad_pic_set_particles. */
int ad_pic_set_particles(ad_pic* h, const double* state);
int ad_pic_get_particles(const ad_pic* h, double* state);
/* The same upload from FP32 host data [6][N][C] for an AD_PIC_FP32_MIXED
   handle: the device state is the same as ad_pic_set_particles gives for the
   FP64 values of these floats, with half the bytes over the host link (C ==
   its padded record size: one copy straight into the state). An FP64 handle
   returns AD_PIC_ERR_UNSUPPORTED. */
int ad_pic_set_particles_f32(ad_pic* h, const float* state);
/* Asynchronous form of ad_pic_set_particles_f32, for streaming many beams
   through one handle (the next beam's upload overlaps the current run).
   ad_pic_prefetch_particles_f32 enqueues the copy of FP32 host data [6][N][C]
   into a device buffer the handle allocates on first use (6 N C floats), on a
   copy stream of its own, and returns without waiting for it. The copy starts
   after the previous commit has read that buffer; a second prefetch before a
   commit replaces the first. The caller keeps the host buffer unchanged until
   the copy is done: until the next ad_pic_run, ad_pic_get_particles or
   ad_pic_destroy returns after ad_pic_commit_particles (pinned host memory
   makes the copy asynchronous; pageable memory is copied before the call
   returns). ad_pic_commit_particles makes the prefetched data the particle
   state, exactly as ad_pic_set_particles_f32 of the same data (kick counter
   and moment history reset), ordered on the handle's stream after the copy,
   without host synchronisation. Commit without a pending prefetch returns
   AD_PIC_ERR_STATE; an FP64 handle returns AD_PIC_ERR_UNSUPPORTED from both. */
int ad_pic_prefetch_particles_f32(ad_pic* h, const float* state);
int ad_pic_commit_particles(ad_pic* h);

/* Set the lattice and recompute the per-kick dual map coefficients (FP64 on
   the host, Eqs. 1-4 applied to the quad matrices of Sec. 4). */
int ad_pic_set_lattice(ad_pic* h, const ad_pic_lattice* lattice);

/* Advance n_steps >= 0 space-charge kicks (each M1(tau/2) M2(tau) M1(tau/2)),
   continuing the kick counter; moments are reduced at every period end and
   after the last kick. Synchronizes before returning; returns
   AD_PIC_ERR_OUT_OF_GRID / _NONFINITE if a kernel flagged a particle, and
   AD_PIC_ERR_TIMEOUT if the push gave up a bounded wait for a state tile
   (the particle state is then not valid: ad_pic_run and ad_pic_get_particles
   return AD_PIC_ERR_STATE until ad_pic_set_beam with normals,
   ad_pic_set_particles or ad_pic_load sets it again). The host-side fault
   injection of the failure tests (no GPU fault) reads the environment:
   ADPIC_FAULT=launch makes the run's launch fail (AD_PIC_ERR_CUDA, nothing
   advanced); ADPIC_FAULT=alloc:K makes every device allocation of a handle
   after its first K fail (AD_PIC_ERR_OOM). */
int ad_pic_run(ad_pic* h, int n_steps);

/* Checkpoint and resume (Sec. 4's periodic-lattice runs are long; a run must
   survive a restart). ad_pic_save writes the dual particle state in the
   handle's precision with the caller's index of every particle, the kick
   counter, the lattice, the reference-particle constants and the moment
   history to `path` (synchronizes the handle's stream; AD_PIC_ERR_STATE if
   no particles are set, AD_PIC_ERR_IO if the file cannot be written).
   ad_pic_load reads such a file into a handle created with the same grid,
   particle count, n_deriv and precision (AD_PIC_ERR_INVALID_ARG otherwise);
   a following ad_pic_run continues the saved run. A failed load leaves the
   handle without particles (AD_PIC_ERR_STATE until they are set). The format
   is the library's own, native byte order. */
int ad_pic_save(const ad_pic* h, const char* path);
int ad_pic_load(ad_pic* h, const char* path);

/* Poll limit of the push's waits for a bulk-copied state tile: polls >= 0
   sets it (0: a wait gives up at once, without polling), polls < 0 restores
   the default of 2^18 polls (each failed poll suspends for a system-dependent
   time, about 1.9 us on GB300, so about half a second). When a wait runs out
   the push records a timeout, lets its copies in flight land (those waits
   keep the default limit) and returns; ad_pic_run then reports
   AD_PIC_ERR_TIMEOUT. A zero limit is how the failure tests make a wait run
   out. Drops captured graphs. */
int ad_pic_set_wait_limit(ad_pic* h, int polls);

/* Device time of a bounded wait that runs out: one thread polls a
   shared-memory barrier that nothing arrives on, `polls` times, on the
   current device's default stream. *ms = its CUDA-event time, *failed = the
   polls that failed (all of them). Allocates 4 bytes of device memory. */
int ad_pic_wait_probe(int polls, double* ms, int* failed);

/* Emittances of the latest moment record: values[2] = (eps_x, eps_y),
   geometric rms (m rad), centred moments; derivs[2*n_deriv] row-major
   d eps_x / d p_k then d eps_y / d p_k. */
int ad_pic_moments(const ad_pic* h, double* values, double* derivs);

/* Raw dual moments of the latest record, mom[3][5][C]: per plane (x, y, z)
   the means <u>, <p>, <u^2>, <u p>, <p^2> over particles (FP64). */
int ad_pic_moments_full(const ad_pic* h, double* mom);

/* Number of moment records kept since the last set_beam/set_particles and
   a copy of them, hist[n][3][5][C]; record 0 is the initial state. */
int ad_pic_history(const ad_pic* h, double* hist, int max_records, int* n_records);

/* Use an external CUDA stream (a cudaStream_t passed as void*); NULL returns
   to the handle's own stream. Drops captured graphs. */
int ad_pic_set_stream(ad_pic* h, void* stream);

/* Capture each distinct run shape in a CUDA graph and replay it (default on). */
int ad_pic_set_graphs(ad_pic* h, int enable);

/* Per-kernel device timing with CUDA events recorded on the handle's stream
   around every launch of the selected kernel classes (bit i = class i, see
   ad_pic_kernel_name). ad_pic_timing returns per class the accumulated
   milliseconds and launch counts since the mask was last set; setting the
   same mask again only resets the accumulators. */
int ad_pic_set_timing(ad_pic* h, unsigned mask);
int ad_pic_timing(const ad_pic* h, double* ms, int64_t* launches, int n_classes);
const char* ad_pic_kernel_name(int cls);
int ad_pic_kernel_classes(void);

/* Kernels launched by ad_pic_run on this handle so far (graph replays count
   every kernel node they run). */
int ad_pic_launches(const ad_pic* h, int64_t* n);

/* Run one stage of the step on the current state and copy its output, for
   parity tests. stage 0: grid geometry, out[6] = origin x,y,z (m), h x,y,z
   (lab, m); 1: deposit, out[C][nz][ny][nx] node charges (C); 2: potential,
   out[C][nz][ny][nx] (V); 3: field, out[3][C][nz][ny][nx] rest-frame V/m;
   4: gather+kick M2(tau) of kick index `kick` with no map, particles updated
   in place (out unused). Stages 1-4 use the geometry of the current state. */
int ad_pic_stage(ad_pic* h, int stage, int64_t kick, double* out);

/* ---------------------------------------------------------------------
   Batched runs: many instances (own lattice, beam, particle count and cubic
   grid each; n_deriv 7) advanced together, as sensitivity scans and line
   searches need. Each kick of every instance is the same split step as
   ad_pic_run; the batch walks it phase by phase for all instances at once in
   one persistent cooperative kernel (or one launch per phase), captured in a
   CUDA graph. All instances must share the kicks per element and be set up
   (beam, lattice) before ad_pic_batch_run; they advance in lockstep.
   --------------------------------------------------------------------- */
typedef struct ad_pic_batch ad_pic_batch;

/* grids[i]: cubic, nx = ny = nz = 32 or 64; n_particles[i] in [1, 2^31 - 1];
   n_deriv must be 7 and precision AD_PIC_FP32_MIXED (else
   AD_PIC_ERR_UNSUPPORTED). Allocates every instance. */
int ad_pic_batch_create(int n_inst, const ad_pic_grid* grids, const int64_t* n_particles, int n_deriv,
                        int precision, ad_pic_batch** out);
/* Per-instance set-up and read-back; same arguments and semantics as the
   single-instance calls (inst in [0, n_inst)); a beam with the bunch charge
   as an AD variable (charge_deriv_slot >= 0) is AD_PIC_ERR_UNSUPPORTED here. */
int ad_pic_batch_set_beam(ad_pic_batch* b, int inst, const ad_pic_beam* beam, const double* normals);
int ad_pic_batch_set_particles(ad_pic_batch* b, int inst, const double* state);
int ad_pic_batch_set_lattice(ad_pic_batch* b, int inst, const ad_pic_lattice* lattice);
int ad_pic_batch_moments(const ad_pic_batch* b, int inst, double* values, double* derivs);
int ad_pic_batch_history(const ad_pic_batch* b, int inst, double* hist, int max_records, int* n_records);
int ad_pic_batch_get_particles(const ad_pic_batch* b, int inst, double* state);
/* Advance every instance n_steps kicks (synchronises). Returns
   AD_PIC_ERR_STATE if the instances are not in lockstep or not set up. */
int ad_pic_batch_run(ad_pic_batch* b, int n_steps);
/* Execution mode: 0 autotune (default; times one kick of the batch in each
   mode on the first run and keeps the fastest), 1 persistent kernel with one
   block per SM, 2 persistent with two, 3 one launch per phase. */
int ad_pic_batch_set_mode(ad_pic_batch* b, int mode);
/* Mode in use and the tuner's per-kick times ms[3] for modes 1..3 (ms; -1 =
   not possible on this device, 0 = not tuned). */
int ad_pic_batch_tuning(const ad_pic_batch* b, int* mode, double* ms);
/* Tile shapes of the batched jobs whose work split is free: tiles[4] =
   (virtual blocks per instance of the moment pass, of the channel maxima, of
   the charge-grid clear, 256-thread field blocks per field virtual block).
   The autotuner (mode 0) picks them after the execution mode by a coordinate
   search, each shape in turn over (4, 8, 16, 32), (2, 4, 8, 16), (4, 8, 16,
   32), (2, 4, 8, 16) with the others held, timing one kick of the real batch
   per choice, and caches them with the mode per batch composition.
   ad_pic_batch_set_tiles fixes them (NULL hands them back to the tuner;
   ranges 1..1024, 1..64, 1..64 and one of 2, 4, 8, 16, else
   AD_PIC_ERR_INVALID_ARG) and makes the next run tune the mode again.
   ad_pic_batch_tiles reads the shapes in use and the tuned kick time in ms
   (0 if not tuned). */
int ad_pic_batch_set_tiles(ad_pic_batch* b, const int* tiles);
int ad_pic_batch_tiles(const ad_pic_batch* b, int* tiles, double* ms);
int ad_pic_batch_set_stream(ad_pic_batch* b, void* stream);
void ad_pic_batch_destroy(ad_pic_batch* b);

/* ---------------------------------------------------------------------
   Learned surrogate (the paper has no counterpart; it warm-starts the
   variable-metric design search of Sec. 3 and Sec. 4): an MLP
   n_in -> width (x hidden layers, GELU) -> n_out trained with the Sobolev
   loss L = 1/B sum_b [ sum_o (y_bo - t_bo)^2 + lambda sum_o,k (dy_bok/dx_k -
   dt_bok)^2 ] on values and derivatives. BF16 weights and activations, FP32
   accumulation on tensor cores, FP32 master weights and Adam.
   Parameters are one flat FP32 vector: for each layer W [out][in] then b [out].
   Host arrays: x [B][n_in], y/t [B][n_out], dy/dt [B][n_out][n_in].
   --------------------------------------------------------------------- */
typedef struct ad_pic_mlp ad_pic_mlp;

/* 1 <= n_in, n_out <= 64; 1 <= width <= 4096; 1 <= hidden <= 16; max_batch B
   with B (n_in + 1) <= 2^24. Parameters start at zero. */
int ad_pic_mlp_create(int n_in, int width, int hidden, int n_out, int max_batch, ad_pic_mlp** out);
int ad_pic_mlp_num_params(const ad_pic_mlp* m, int64_t* n);
/* Set (resets the Adam moments) / read the FP32 parameter vector. */
int ad_pic_mlp_set_params(ad_pic_mlp* m, const float* params);
int ad_pic_mlp_get_params(const ad_pic_mlp* m, float* params);
/* Values y and, if dy is not NULL, input derivatives (forward mode). */
int ad_pic_mlp_forward(ad_pic_mlp* m, const float* x, int B, float* y, float* dy);
/* Sobolev loss and (if grad is not NULL) its gradient w.r.t. the flat parameters. */
int ad_pic_mlp_loss_grad(ad_pic_mlp* m, const float* x, const float* t, const float* dt, int B, float lambda,
                         double* loss, float* grad);
/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8) on the Sobolev loss of the batch;
   *loss is the loss before the step. */
int ad_pic_mlp_adam_step(ad_pic_mlp* m, const float* x, const float* t, const float* dt, int B, float lambda, float lr,
                         double* loss);
/* Device-resident training. ad_pic_mlp_set_dataset uploads n samples (x
   [n][n_in], t [n][n_out], dt [n][n_out][n_in], host, already in the order
   the mini-batches should take them) once. ad_pic_mlp_train then runs
   `steps` Adam steps of B samples each (consecutive samples of the set,
   wrapping around) with the Sobolev loss of weight lambda and the learning
   rate lr0 (lr1/lr0)^(s/(steps-1)) at step s: every step is one replay of a
   CUDA graph (batch gather, forward and tangent GEMMs, loss, backward, Adam)
   with its counters on the device, so no host transfer or synchronisation
   happens between steps. *loss receives the last step's loss (before its
   update), *ms the CUDA-event time of the steps (either may be NULL). Adam's
   step count carries over from ad_pic_mlp_adam_step and earlier runs.
   AD_PIC_ERR_STATE without a dataset. */
int ad_pic_mlp_set_dataset(ad_pic_mlp* m, const float* x, const float* t, const float* dt, int n);
int ad_pic_mlp_train(ad_pic_mlp* m, int steps, int B, float lambda, float lr0, float lr1, double* loss, double* ms);
void ad_pic_mlp_destroy(ad_pic_mlp* m);

/* Allocation-free dual moments of a caller-owned device state (the paper has
   no counterpart: this exists for callers that cannot let the library call
   cudaMalloc/cudaFree - code running inside another framework's device-memory
   budget, or latency-critical loops that must not take the implicit
   synchronisation those calls can bring).
   state_dev: device pointer to the dual state [6][n_particles][CP] of the
   precision's type (double for AD_PIC_FP64, float for AD_PIC_FP32_MIXED),
   CP = 8 for n_deriv 7 and 16 for n_deriv 13 (channels beyond n_deriv+1 are
   padding). mom_dev: device pointer to 15*CP doubles, written as
   [3][5][CP] per plane (x, y, z) the means <u>, <p>, <u^2>, <u p>, <p^2>.
   stream: cudaStream_t as void* (NULL = default stream); the call only
   enqueues work and does not synchronise. The per-block partial sums live in
   one static device array of 583,680 bytes (304 blocks x 15 x 16 doubles)
   that every GPU loading the library holds until exit. n_deriv must be 7 or
   13 (AD_PIC_ERR_INVALID_ARG otherwise): only those two channel layouts are
   compiled; the array holds up to 16 channels. Every call made outside
   stream capture looks the array's address up (cudaGetSymbolAddress) with
   the current device; a call made while `stream` is capturing uses the
   address of the last such lookup on that device, so make a first call on
   each device before any stream capture (AD_PIC_ERR_STATE otherwise). If a
   CUDA error is already pending at entry, the call returns AD_PIC_ERR_CUDA
   without launching and leaves that error pending. All calls share the
   array, so calls that overlap on the GPU race. */
int ad_pic_moments_device(const void* state_dev, int64_t n_particles, int n_deriv, int precision, double* mom_dev,
                          void* stream);

/* Measured fused multiply-add throughput of the current device (the ALU
   ceiling of the plain FP64 path and of the FP32 arithmetic of the mixed
   path, which the paper does not state): precision AD_PIC_FP32_MIXED times
   FP32 FMA chains, AD_PIC_FP64 FP64 FMA chains, 8 independent chains per
   thread on 8 blocks of 256 threads per SM, best of 5 CUDA-event-timed
   launches after a warm-up; *tflops counts an FMA as 2 flops. Changes no
   device setting; allocates a small output buffer. */
int ad_pic_fma_peak(int precision, double* tflops);

/* ---------------------------------------------------------------------
   Single-particle dual optics (Sec. 3): beamlines of drifts and thick
   quadrupoles whose lengths and strengths may be AD variables. FP64.
   --------------------------------------------------------------------- */
enum { AD_PIC_DRIFT = 0, AD_PIC_QUAD = 1 };

/* One element. k is the normalised strength (1/m^2) of a quadrupole: the
   thick-lens matrix of Sec. 4, Eq. "quadtr" (cos/sin with sqrt(k) in the
   focusing plane, cosh/sinh in the other), focusing in x for k > 0. slot_L
   and slot_k are derivative slots (0 .. n_deriv-1) or -1 for a constant. */
typedef struct {
    int type;          /* AD_PIC_DRIFT or AD_PIC_QUAD */
    int slot_L, slot_k;
    int pad;
    double L;          /* length (m), >= 0 */
    double k;          /* strength (1/m^2), quadrupoles only */
} ad_pic_element;

/* Twiss functions at the end of n_inst beamlines of n_elem elements each
   (elems [n_inst][n_elem], host), with derivatives w.r.t. n_deriv <= 15
   slots: out [n_inst][4][n_deriv+1] = (beta_x, alpha_x, beta_y, alpha_y),
   value then derivatives. If n_cell > 0 the start values are the periodic
   Twiss functions of the first n_cell elements of the instance (cos mu =
   (m11 + m22)/2, beta = m12 / sin mu, alpha = (m11 - m22) / (2 sin mu),
   sin mu with the sign of m12; dual, so they carry derivatives too) and the
   transport (Sec. 3, Eq. 5) runs through the remaining elements; if n_cell
   is 0 the start values are the constants twiss0 [n_inst][4] and the
   transport runs through all elements. One GPU thread per instance.
   AD_PIC_ERR_UNSTABLE if a cell has no periodic solution (that instance's
   output is not valid). Allocates and frees device buffers per call. */
int ad_pic_twiss_batch(int n_inst, int n_elem, const ad_pic_element* elems, int n_deriv, int n_cell,
                       const double* twiss0, double* out);

/* A general beamline in place of the FODO period of ad_pic_set_lattice (the
   matching-section runs of Sec. 4): n_elem elements in beam order, kicks[e]
   >= 1 space-charge kicks in element e (each M1(tau/2) M2(tau) M1(tau/2)
   with tau = L / kicks, Sec. 4), quadrupole strengths k (1/m^2) and lengths
   as dual variables through their slots (< n_deriv, or -1). The kick
   schedule and the moment records then follow the beamline: one record at
   the end of every pass. Lengths > 0. Replaces any lattice set before;
   ad_pic_set_lattice replaces the beamline. Drops captured graphs. */
int ad_pic_set_beamline(ad_pic* h, int n_elem, const ad_pic_element* elems, const int* kicks);

/* Element-by-element tracking of n_part particles x0 [n_part][4] (x, px, y,
   py; host) through the beamline repeated n_repeat times (turns x periods),
   with derivatives w.r.t. n_deriv <= 32 slots: out [n_part][4][n_deriv+1]
   (host). FP64; every derivative channel follows d(M z) = M dz + (dM) z with
   the element maps M computed once on the host (dual FP64). One GPU thread
   per particle and chunk of 8 derivative channels; the maps of all elements
   sit in shared memory (AD_PIC_ERR_UNSUPPORTED beyond 200 KB). If ms is not
   NULL it receives the kernel's CUDA-event time. Allocates and frees device
   buffers per call. */
int ad_pic_track_batch(int64_t n_part, const double* x0, int n_elem, const ad_pic_element* elems, int n_deriv,
                       int64_t n_repeat, double* out, double* ms);

/* ---------------------------------------------------------------------
   2D dual PIC in a rectangular, perfectly conducting pipe (Sec. 4, the
   paper's own solver): a coasting beam with coordinates (x, px, y, py) as
   dual numbers; bilinear deposit of the normalised density on nx x ny cells
   of the a x b pipe (nodes 0..nx, 0..ny, the walls at 0 and n, the beam axis
   at the centre); Poisson's equation with phi = 0 on the walls by the sine
   series of Sec. 4 (rho^lm = (4/(nx ny)) sum rho_ij sin(l pi i/nx) sin(m pi
   j/ny), phi^lm = rho^lm / gamma_lm^2, gamma_lm^2 = (l pi/a)^2 + (m pi/b)^2,
   sine sums back); central-difference fields (zero on the walls); the kick
   p += 2 pi K E tau of H2 = K phi / 2 with K = q I / (2 pi eps0 p0 v0^2
   gamma0^2) and phi normalised to unit charge; the FODO maps of
   ad_pic_set_lattice in x and y. A particle within one cell of a wall is
   flagged (AD_PIC_ERR_OUT_OF_GRID, index clamped).
   --------------------------------------------------------------------- */
typedef struct ad_pic2d ad_pic2d;

/* nx, ny in [8, 512] cells, a, b > 0 (m), n_particles in [1, 2^31 - 1],
   n_deriv 7 or 13, precision AD_PIC_FP64 or AD_PIC_FP32_MIXED. */
int ad_pic2d_create(int nx, int ny, double a, double b, int64_t n_particles, int n_deriv, int precision,
                    ad_pic2d** out);
/* Reference particle and Twiss functions of the x and y planes from `beam`
   (z ignored), the beam current I (A) and its derivative slot (or -1). If
   normals is not NULL it is [4][N] standard-normal draws (n1, n2 of x, then
   y): u = sqrt(eps beta) n1, p = sqrt(eps/beta)(n2 - alpha n1), eps =
   eps_n / (beta0 gamma0), sample mean removed. */
int ad_pic2d_set_beam(ad_pic2d* h, const ad_pic_beam* beam, double current_A, int current_deriv_slot,
                      const double* normals);
/* state [4][N][n_deriv+1] (host FP64) */
int ad_pic2d_set_particles(ad_pic2d* h, const double* state);
int ad_pic2d_get_particles(const ad_pic2d* h, double* state);
int ad_pic2d_set_lattice(ad_pic2d* h, const ad_pic_lattice* lattice);
/* n_steps kicks M1(tau/2) M2(tau) M1(tau/2); moments at period ends and after the last kick */
int ad_pic2d_run(ad_pic2d* h, int n_steps);
/* emittances (x, y) of the latest record and derivs [2][n_deriv]; raw moments [2][5][C]; history [n][2][5][C] */
int ad_pic2d_moments(const ad_pic2d* h, double* values, double* derivs);
int ad_pic2d_moments_full(const ad_pic2d* h, double* mom);
int ad_pic2d_history(const ad_pic2d* h, double* hist, int max_records, int* n_records);
void ad_pic2d_destroy(ad_pic2d* h);

/* Derived constants: out[8] = gamma0, beta0, p0 (kg m/s), B rho (T m),
   kappa_perp, kappa_z (1/(V/m * m)), macroparticle charge (C), q (C). */
int ad_pic_constants(const ad_pic* h, double* out);

void ad_pic_destroy(ad_pic* h);
const char* ad_pic_strerror(int status);

#ifdef __cplusplus
}
#endif
#endif
