/*
 * lbem.h -- C ABI of the GB300 (sm_103a) lattice-Boltzmann electromagnetic
 * scattering library: the D3Q7 vector-population LB scheme for Maxwell's
 * equations of arXiv 2510.11042 (Sec. 2), with a total-field/scattered-field
 * plane-wave source, an absorbing outer layer, a running single-frequency DFT
 * of the near fields and the near-to-far-field projection of the angular
 * scattering intensity |S|^2 (Eqs. 5-10).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Units: lattice units, dx = dt = 1, vacuum speed of light c = 1/3 (Sec. 2.1,
 * Eq. 3), vacuum impedance one, wavenumber k = 2 pi / lambda, period
 * T = 3 lambda steps.  Angles are radians.
 *
 * Status: every function returning int32_t returns LBEM_OK (0) or a negative
 * LBEM_ERR_* code; no C++ exception crosses this boundary.  The text of the
 * last error of a handle is available from lbem_last_error().  A failed call
 * leaves the handle's state as it was, except lbem_step(), after which the
 * handle holds whatever steps completed before the failure.
 *
 * Streams and threads: a handle is bound to the CUDA stream given at creation
 * (NULL = the legacy default stream) and to the current device at that moment.
 * Calls on one handle must not race; different handles are independent.
 * Every call that returns results to the host synchronises the stream; the
 * others only enqueue work.
 *
 * Memory: pointers named *_host are host memory (pageable or pinned), pointers
 * named *_dev are device memory of the handle's device; arguments with an
 * "on_device" flag accept either.  The library never keeps a caller pointer
 * beyond a call, except the workspace passed to lbem_create(), which the
 * caller must keep alive until lbem_destroy().
 *
 * Population layout (lbem_get_populations / lbem_set_populations):
 * float32 [Q][nz][ny][nx], plane q = (family, direction i, component a),
 * families e then h (Sec. 2.1: e_i, h_i), directions i = 0..6 in the order
 * c_0 = 0, +x, -x, +y, -y, +z, -z, and per family only the components the
 * mode carries:
 *   LBEM_MODE_EZ (2D, E along z; "TM" for cylinders, Sec. 3.2): e_z; h_x, h_y  (Q = 21)
 *   LBEM_MODE_HZ (2D, H along z; "TE"):                         e_x, e_y; h_z  (Q = 21)
 *   LBEM_MODE_3D:                                               e_xyz; h_xyz   (Q = 42)
 * e.g. in EZ mode q = i for e_z of direction i, q = 7 + 2 i + a for h_a.
 * A 2D grid has nz == 1 and is periodic along z (the +-z populations stream
 * onto themselves).  The stored populations are the post-collision ones.
 */
#ifndef LBEM_H
#define LBEM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    LBEM_OK = 0,
    LBEM_ERR_ARG = -1,       /* invalid argument, shape, box or polarisation */
    LBEM_ERR_OOM = -2,       /* device allocation failed or workspace too small */
    LBEM_ERR_CUDA = -3,      /* a CUDA runtime call or kernel launch failed */
    LBEM_ERR_NONFINITE = -4, /* a NaN or Inf was found in the state */
    LBEM_ERR_TIMEOUT = -5,   /* a bounded wait ran out */
    LBEM_ERR_STATE = -6      /* call not valid in the handle's state */
};

typedef struct lbem_ctx *lbem_handle;

/* The only velocity set of the paper: D3Q7 (Sec. 2.1). */
typedef enum { LBEM_D3Q7 = 0 } lbem_velocity_set;

/* Storage type of the populations in device memory.  The update arithmetic is
 * float32 in every case; F16/BF16 store populations divided by one power-of-two
 * scale (see lbem_set_storage_scale) and round to nearest even.  Inside the
 * total-field box the stored values are the scattered part (the total minus
 * the incident line's populations), elsewhere the scattered field itself, so
 * the storage rounding error is relative to the scattered field. */
typedef enum { LBEM_F32 = 0, LBEM_F16 = 1, LBEM_BF16 = 2 } lbem_storage;

typedef enum { LBEM_MODE_EZ = 0, LBEM_MODE_HZ = 1, LBEM_MODE_3D = 2 } lbem_mode;

/* The lattice.  nz == 1 with an EZ/HZ mode is a 2D problem; LBEM_MODE_3D needs
 * nz >= 2.  absorber_width W cells on every face of an axis longer than one
 * cell: post-collision populations are multiplied by 1 - sigma_max (m/W)^3,
 * m = W - d, d = distance in cells to the nearest such face (the paper's
 * outer boundary, Sec. 2.2, Eq. 4, is the clamped pull at the faces; the
 * layer itself is this library's reading of the absorbing layers the paper
 * names as future work, Sec. 4).  sigma_max <= 0 selects 0.3. */
typedef struct {
    int32_t nx, ny, nz;
    int32_t absorber_width;
    double sigma_max;
    int32_t storage;    /* lbem_storage */
    int32_t mode;       /* lbem_mode */
    int32_t streaming;  /* lbem_streaming (0: two buffers) */
} lbem_grid_desc;

/* How the populations stream between steps (the pull step of Sec. 2.1 with
 * the Eq. 4 clamp in either case; the same populations bit for bit):
 *  LBEM_STREAM_TWO_BUFFERS: read one population buffer, write the other; the
 *    default, and the only scheme with two-step passes (lbem_set_step_fusion),
 *    batched runs and the adjoint.
 *  LBEM_STREAM_IN_PLACE: one buffer (half the population memory, so larger
 *    grids fit) updated in place by alternating a step that pushes each
 *    post-collision population into its downstream neighbour's opposite slot
 *    and a step that reads and writes only the cell's own slots (the "AA"
 *    pattern), with thin face buffers (four per axis longer than one cell) for
 *    the clamped faces of Eq. 4.
 *    Single steps only.  The state is in its ordinary layout after an even
 *    number of steps; calls that read or set populations or fields after an
 *    odd number first rearrange it (one pass over the populations).
 *    lbem_batch_create, lbem_forward_checkpointed and lbem_adjoint refuse such
 *    handles with LBEM_ERR_ARG. */
typedef enum { LBEM_STREAM_TWO_BUFFERS = 0, LBEM_STREAM_IN_PLACE = 1 } lbem_streaming;

/* A linearly polarised incident plane wave (Sec. 2.3: "the incident field
 * considered in this work is linearly polarized").  dir must be +x or +y for
 * the 2D modes and +x, +y or +z in 3D; pol must be a unit vector orthogonal to
 * dir (along z for EZ, in the xy plane for HZ).  The incident field is
 * E(t) = amplitude * ramp(t) * sin(w t) * pol, H = dir x E, ramp a raised
 * cosine over ramp_periods periods, w = 2 pi / T, T = 3 * wavelength, which
 * must be an integer.  It is carried by a 1D D3Q7 line along dir that shares
 * the grid's coordinate along dir, is driven at node source_index (-1: W + 2)
 * and has the same absorbing layer at both ends; every lattice link that
 * crosses the surface of the total-field box [tfsf_lo, tfsf_hi] (inclusive
 * cell indices) adds (entering) or subtracts (leaving) the line's incident
 * population of the link's source cell.  The NTFF box [ntff_lo, ntff_hi] must
 * enclose the total-field box strictly and lie outside the absorbing layer;
 * center is the phase reference of the far field.  For 2D grids the z entries
 * of the boxes must be 0.
 *
 * source_kind = LBEM_SOURCE_ANALYTIC instead takes the incident populations
 * from the closed-form plane wave: the vacuum equilibrium (Eq. 2) of
 * E = amplitude * ramp(tau) * sin(w tau) * pol, H = dir x E at the link's
 * source cell r and time n, tau = n - 3 dir.(r - origin) (c = 1/3, Eq. 3).  dir
 * may then be any unit vector (in the xy plane for the 2D modes), and the
 * total-field box may extend past the grid (a one-sided box, e.g. the
 * half-space x >= x_s) and into the absorbing layer.  An NTFF box is then
 * optional: all-zero ntff bounds mean none (no DFT, no far field), otherwise
 * the rules above apply and |E_I| of Eqs. 5-6 is the amplitude.  The
 * analytic wave is not an exact solution of the discrete scheme, so every
 * cell of the total-field box carries a source term; the line source is
 * exact and costs nothing outside dielectric cells. */
#define LBEM_SOURCE_LINE 0
#define LBEM_SOURCE_ANALYTIC 1
typedef struct {
    double dir[3];
    double pol[3];
    double wavelength;
    double amplitude;
    double ramp_periods;
    int32_t tfsf_lo[3], tfsf_hi[3];
    int32_t ntff_lo[3], ntff_hi[3];
    double center[3];
    int32_t source_index;
    int32_t source_kind;   /* LBEM_SOURCE_LINE or LBEM_SOURCE_ANALYTIC */
    double origin[3];      /* analytic source: where tau = n */
} lbem_plane_wave;

/* Bytes of device workspace a grid needs (populations in two buffers, or one
 * with the face buffers of in-place streaming, the permittivity map, the
 * incident line, the DFT accumulators and scratch). */
int32_t lbem_workspace_bytes(const lbem_grid_desc *grid, size_t *bytes_out);

/* Create a solver on the current device.
 * eps_r: relative permittivity per cell, float32 [nz][ny][nx], values >= 1
 *   (non-absorbing dielectrics, Sec. 2.1; mu_r = 1 as in all of the paper's 2D
 *   and 3D work, Sec. 3.1), host or device memory (eps_on_device).  Copied.
 * cuda_stream: cudaStream_t the handle enqueues on (NULL: legacy default stream).
 * workspace: device memory of at least lbem_workspace_bytes(), 256-byte
 *   aligned, owned by the caller; NULL makes the library cudaMalloc it and
 *   free it in lbem_destroy().
 * The populations start at zero (vacuum, no field). */
int32_t lbem_create(const lbem_grid_desc *grid, int32_t velocity_set, const float *eps_r,
                    int32_t eps_on_device, void *cuda_stream, void *workspace,
                    size_t workspace_bytes, lbem_handle *out);

/* Replace the permittivity map (same layout and rules as in lbem_create). */
int32_t lbem_set_permittivity(lbem_handle h, const float *eps_r, int32_t eps_on_device);

/* Attach an incident plane wave (see lbem_plane_wave).  Resets the incident
 * line to zero; the main lattice keeps its state and its time. */
int32_t lbem_inject_plane_wave(lbem_handle h, const lbem_plane_wave *wave);

/* Record the DFT of the fields over n_periods whole periods starting at field
 * time t_start (Sec. 2.4: "over one period of the steady-state oscillation"):
 * X = 2/(n_periods T) sum_t x(t) exp(-j w t), x the moments computed in the
 * step that produces time t.  Clears the accumulators.  Needs a plane wave. */
int32_t lbem_set_dft_window(lbem_handle h, int64_t t_start, int32_t n_periods);

/* Advance n time steps (Eq. 1 with the equilibria of Eq. 2, streaming with the
 * outer boundary of Eq. 4, the TF/SF source, the absorbing layer and the DFT
 * of the near fields), asynchronously on the handle's stream. */
int32_t lbem_step(lbem_handle h, int64_t n);

/* Number of steps taken since creation (the time of the stored state). */
int32_t lbem_get_time(lbem_handle h, int64_t *t_out);

/* Magnetic media: a per-cell relative permeability map (nx*ny*nz floats, x
 * fastest; host or device), validated like eps_r (finite, >= 1, else
 * LBEM_ERR_ARG with the handle unchanged).  Eq. 2's rest population becomes
 * h_0^eq = (mu_r - 1) H with H = B / mu_r, and the TF/SF source of magnetic
 * cells carries the field H_inc (1/mu_r - 1).  Every step then reads 4 more
 * bytes per cell.  mu_r == NULL returns to mu_r = 1 everywhere.  The paper
 * uses mu_r != 1 only in its 1D interface tests (Sec. 3.1, Eq. 11).  Batched
 * runs and the adjoint support mu_r = 1 only. */
int32_t lbem_set_permeability(lbem_handle h, const float *mu_r, int32_t mu_on_device);

/* Angular scattering intensity |S|^2 (Eqs. 5, 6) by the near-to-far-field
 * projection of Eqs. 7-10 in the far-field limit, from the DFT accumulators:
 * J = n x H, M = -n x E on the NTFF box faces (trapezoidal rule per face),
 * N = sum w J exp(j k r_hat.(r'-center)), L likewise with M;
 *   3D: |S|^2 = k^4 (|N_th + L_ph|^2 + |N_ph - L_th|^2) / (16 pi^2 |E_I|^2),
 *       r_hat = (sin th cos ph, sin th sin ph, cos th);
 *   EZ: |S|^2 = k^2 |N_z - L_ph|^2 / (8 pi |E_I|^2),
 *   HZ: |S|^2 = k^2 |N_ph + L_z|^2 / (8 pi |E_I|^2),  r_hat = (cos th, sin th, 0);
 * |E_I| the incident line's E phasor along pol at the centre (Eq. 5/6: "in the
 * vicinity of the scatterer").  theta_host, phi_host: n angles (phi ignored
 * and may be NULL in 2D).  s2_host: n outputs.  amp_host (optional, NULL): 12
 * doubles per angle, Re/Im of N_x, N_y, N_z, L_x, L_y, L_z.  Inputs and
 * outputs are FP64.  In 2D the projection is FP64 throughout; in 3D it is a
 * complex FP32 contraction (phasors and FP64-evaluated phases rounded once to
 * FP32, FP32 sums over at most a chunk of face rows and a 64-column tile, FP64
 * sums above), deterministic call to call. */
int32_t lbem_far_field(lbem_handle h, const double *theta_host, const double *phi_host,
                       int32_t n, double *s2_host, double *amp_host);

/* Temporal blocking (Eq. 1 applied twice per pass over memory):
 * steps_per_pass = 2 (the default) lets lbem_step advance grids of any mode
 * and storage, with or without a mu_r map, two steps per pass over the
 * populations: a fused kernel keeps the intermediate state of each tile (3D:
 * 32 x 8 cells in FP32, 32 x 16 in FP16/BF16, marching through a chunk of z
 * planes; 2D: 128-cell strips marching along y) plus its edge halos in shared
 * memory, bitwise the same result as two single steps (16-bit storage rounds
 * the intermediate state as a single step stores it).  It is taken where its
 * blocks fill the GPU (one wave of resident blocks in 3D, two in 2D) and, in
 * 2D, where the population buffers of the grids stepping together outgrow
 * the L2 cache (smaller grids are served from it); other grids, the
 * closed-form source (bound by its wave evaluations, not by memory), a last
 * odd step and handles with in-place streaming take single steps.
 * 1 always takes single steps.  Anything else: LBEM_ERR_ARG. */
int32_t lbem_set_step_fusion(lbem_handle h, int32_t steps_per_pass);

/* The steps per pass lbem_step takes on this handle as it is now configured:
 * 2 where two-step passes apply (see lbem_set_step_fusion), else 1.
 * NULL argument: LBEM_ERR_ARG. */
int32_t lbem_get_step_fusion(lbem_handle h, int32_t *steps_per_pass);

/* Precision of the 3D projection in lbem_far_field (2D is always FP64).
 * LBEM_FAR_FIELD_MIXED (the default): the FP32 contraction described above.
 * LBEM_FAR_FIELD_FP64: FP64 products and sums throughout, ~30x slower on
 * GB300 (its FP64 pipe runs at 1/64 of the FP32 rate).  Anything else:
 * LBEM_ERR_ARG with the setting unchanged. */
#define LBEM_FAR_FIELD_MIXED 0
#define LBEM_FAR_FIELD_FP64 1
int32_t lbem_set_far_field_precision(lbem_handle h, int32_t precision);

/* |E_I| as used by lbem_far_field. */
int32_t lbem_incident_amplitude(lbem_handle h, double *out_host);

/* Field probes: the Q total-field populations (the stored value plus, inside
 * the total-field box, the incident part) of n listed cells, at the stored
 * state's time.  xyz_host: n (x, y, z) triplets inside the grid; out_host:
 * n * Q floats, out[k * Q + q] in the population-plane order above.
 * n <= LBEM_PROBE_MAX, else LBEM_ERR_ARG; a cell outside the grid is
 * LBEM_ERR_ARG.  Synchronous. */
#define LBEM_PROBE_MAX 4096
int32_t lbem_probe(lbem_handle h, const int32_t *xyz_host, int32_t n, float *out_host);

/* Copy the populations out / in, float32 [Q][nz][ny][nx] (layout above). */
int32_t lbem_get_populations(lbem_handle h, float *out, int32_t out_on_device);
int32_t lbem_set_populations(lbem_handle h, const float *in, int32_t in_on_device);

/* Fields of the stored state, E = sum_i e_i / eps_r, H = sum_i h_i (the zeroth
 * moments of Sec. 2.1), float32 [3][nz][ny][nx] each (components x, y, z). */
int32_t lbem_fields(lbem_handle h, float *E_out, float *H_out, int32_t out_on_device);

/* DFT phasors on the NTFF box faces, FP64.  Faces f = 2*axis + side (side 0 at
 * ntff_lo, 1 at ntff_hi) for each axis longer than one cell, in that order;
 * per face [C][2][nu][nv] (component, re/im, u, v), (u, v) = (z, y) for
 * x-faces, (z, x) for y-faces, (y, x) for z-faces, each spanning the NTFF box.
 * Components C: EZ (E_z, H_x, H_y); HZ (E_x, E_y, H_z); 3D (E_x..H_z).
 * lbem_dft_doubles() gives the total count. */
int32_t lbem_dft_doubles(lbem_handle h, size_t *count_out);
int32_t lbem_get_dft(lbem_handle h, double *out_host);

/* Physical energy 1/2 sum (eps_r |E|^2 + |H|^2) of the stored state (the
 * steady-state monitor of Sec. 3.2), FP64; LBEM_ERR_NONFINITE if any
 * population is NaN or Inf. */
int32_t lbem_energy(lbem_handle h, double *out_host);

/* Checkpoint: opaque snapshot of populations, incident line, DFT accumulators,
 * time and storage scale, for the same grid description (the plane wave and
 * the permittivity are not part of it: set them as for the saved run). */
int32_t lbem_state_bytes(lbem_handle h, size_t *bytes_out);
int32_t lbem_save_state(lbem_handle h, void *buf_host, size_t bytes);
int32_t lbem_load_state(lbem_handle h, const void *buf_host, size_t bytes);

/* Power-of-two scale of the reduced-precision storage, shared by all planes:
 * stored = population / scale (default 2^-10 for F16, 1 for BF16; always 1 for
 * LBEM_F32, where the call is a no-op).  Setting it rescales the stored state.
 * One scale for all planes lets the linear update run in storage units. */
int32_t lbem_set_storage_scale(lbem_handle h, float scale);
int32_t lbem_get_storage_scale(lbem_handle h, float *scale_out);

/* Batched runs (the workload of many uneven scatterers advanced together):
 * a batch groups existing handles of the same mode and storage on one device
 * and advances them in one persistent cooperative launch whose blocks stride
 * over the row tiles of all problems, with a bounded grid barrier between
 * steps.  lbem_batch_run(b, steps, autotune) advances handle i by steps[i]
 * (problems that are done drop out); with autotune the first call times a
 * few candidate launch shapes (blocks per SM, rows per work item) on its
 * first steps, which count as real steps (the results do not depend on the
 * shape), and keeps the fastest.  It then also times split schedules, in
 * which grids of at least 2^k cells (k = 16..20) advance by one plain step
 * launch each (such a grid fills much of the GPU by itself, and the
 * persistent kernel's grid barrier would only add to its step) while the rest
 * share the persistent launch, and keeps one when it is faster
 * (lbem_batch_config's split = 1).  In a split schedule the large grids run
 * on four internal lane streams (problem j on lane j mod 4, in turns of 64
 * steps) forked from and joined back into cuda_stream, so that they overlap;
 * the persistent launch follows them.  autotune = 0 runs everything persistent
 * at the largest resident shape; autotune = 2 forces the split schedule at
 * 2^19 cells without timing.
 * The handles' own streams are synchronised first; the batch runs on
 * cuda_stream and returns when it is done.  LBEM_ERR_TIMEOUT reports a
 * grid-barrier wait that ran out.  workspace: as in lbem_create (NULL: the
 * library allocates it). */
typedef struct lbem_batch_ctx *lbem_batch;
int32_t lbem_batch_workspace_bytes(int32_t count, size_t *bytes_out);
int32_t lbem_batch_create(const lbem_handle *handles, int32_t count, void *cuda_stream,
                          void *workspace, size_t workspace_bytes, lbem_batch *out);
int32_t lbem_batch_run(lbem_batch b, const int64_t *steps, int32_t autotune);
int32_t lbem_batch_config(lbem_batch b, int32_t *blocks_per_sm, int32_t *rows_per_item,
                          double *ms_per_step, int32_t *split);
int64_t lbem_batch_launches(lbem_batch b);
/* Failure-path check of the batched kernel's bounded grid barrier (no
 * counterpart in the paper): one block waits at the barrier for an arrival
 * that never comes.  Its wait gives up after about a second and reports
 * through the status word, as a real stall would; the call then returns
 * LBEM_ERR_TIMEOUT with the same message lbem_batch_run gives, and the batch
 * and its handles stay usable.  Any other return is a fault of the check. */
int32_t lbem_batch_selftest_barrier(lbem_batch b);
const char *lbem_batch_last_error(lbem_batch b);
void lbem_batch_destroy(lbem_batch b);

/* Gradient of far-field intensities with respect to the permittivity map: the
 * discrete adjoint of lbem_step (the paper's scheme is linear in the
 * populations for a fixed eps_r map, so the adjoint of each step is its
 * transpose; the paper itself computes no gradients).  The objective is
 *   J = sum_k weights[k] |S(theta_k, phi_k)|^2     (|S|^2 of lbem_far_field)
 * and the result is dJ/deps_r for every cell, through every step of the run:
 * collision (Eqs. 1-2), clamped streaming (Eq. 4), the TF/SF source, the
 * absorbing layer and the DFT window (|E_I| does not depend on eps_r).
 * FP32 storage only (LBEM_ERR_ARG otherwise).
 *
 * lbem_forward_checkpointed(h, n_steps, K, ...) replaces lbem_step for a run
 * that is to be differentiated: it must start at t = 0 (right after
 * lbem_inject_plane_wave, with the DFT window set) and takes n_steps steps,
 * keeping the state at every K-th step in its workspace
 * (lbem_adjoint_workspace_bytes; NULL: the library allocates it and frees it
 * with the handle).  The workspace holds ceil(n_steps / K) checkpoints of the
 * populations plus K steps of recorded fields (NE floats per cell and step),
 * so K ~ sqrt(n_steps * populations / NE) minimises it.
 *
 * lbem_adjoint then replays each segment forward from its checkpoint and runs
 * the adjoint steps backwards through it: about two more steps' worth of work
 * per step.  theta, phi (phi may be NULL in 2D), weights: n_ang (1..1024) host
 * doubles.  grad_out: nx*ny*nz floats, x fastest, on the device when
 * grad_on_device, else host memory.  J_out (host, optional): the objective.
 * It may be called again with other angles or weights; lbem_set_permittivity,
 * lbem_inject_plane_wave, lbem_set_dft_window, lbem_set_populations and
 * lbem_load_state discard the checkpoints (then LBEM_ERR_STATE).  The DFT
 * window must lie inside the checkpointed steps.  Synchronous. */
int32_t lbem_adjoint_workspace_bytes(lbem_handle h, int64_t n_steps, int32_t K, size_t *bytes_out);
int32_t lbem_forward_checkpointed(lbem_handle h, int64_t n_steps, int32_t K, void *workspace,
                                  size_t workspace_bytes);
int32_t lbem_adjoint(lbem_handle h, const double *theta_host, const double *phi_host,
                     const double *weights_host, int32_t n_ang, float *grad_out,
                     int32_t grad_on_device, double *J_out);
/* Device time (CUDA events on the handle's stream) of the last lbem_adjoint
 * call: the forward replays of all segments and the adjoint steps. */
int32_t lbem_adjoint_timing(lbem_handle h, double *replay_ms, double *backward_ms);

/* Far-field projection that allocates nothing (the paper has no counterpart;
 * this is a library convenience).  For callers that cannot call cudaMalloc or
 * any allocator -- e.g. a host application that owns the device memory budget
 * and gives plugins fixed buffers, or a real-time loop where allocation is not
 * allowed -- it computes the same |S|^2 as lbem_far_field from caller-owned
 * device memory only:
 *   dft_dev   the face phasors in the layout of lbem_get_dft (device copy),
 *   theta_dev, phi_dev (phi ignored, may be NULL, in 2D), n angles,
 *   s2_dev    n outputs; amp_dev optional (NULL), 12 doubles per angle,
 * with |E_I| given in desc (e.g. from lbem_incident_amplitude).  Its only
 * scratch, the partial sums of the projection, lives in a fixed array of
 * LBEM_NOALLOC_MAX_ANGLES x 16 x 12 doubles (1.5 MB) that every GPU loading
 * the library holds until the process exits; n > LBEM_NOALLOC_MAX_ANGLES is
 * rejected with LBEM_ERR_ARG (split larger angle sets over several calls).
 * The first call on a device looks up that array's device address (once per
 * device, with the device current) and keeps it for the process: it assumes
 * the CUDA runtime's primary context of the device and no cudaDeviceReset
 * afterwards.  Make that first call before any stream capture.  All calls
 * share the array, so calls whose work overlaps on the GPU (different streams,
 * or threads) race and must be serialised by the caller.  Every pointer must
 * be device (or managed) memory of the current device, and the caller sizes
 * them: dft_dev as lbem_get_dft lays out desc's NTFF box, theta_dev, phi_dev
 * and s2_dev n doubles, amp_dev 12 n; a host pointer or one of another device
 * is rejected with LBEM_ERR_ARG, sizes cannot be checked here.
 * Asynchronous on cuda_stream (NULL: legacy default stream); errors are
 * reported by the return code and lbem_last_error(NULL). */
#define LBEM_NOALLOC_MAX_ANGLES 1024
typedef struct {
    int32_t mode;                  /* lbem_mode */
    int32_t nx, ny, nz;            /* grid extents (nz == 1 for the 2D modes) */
    int32_t ntff_lo[3], ntff_hi[3];/* NTFF box of the DFT data */
    double wavelength;             /* cells; k = 2 pi / wavelength */
    double center[3];              /* phase reference */
    double incident_amplitude;     /* |E_I| of Eqs. 5-6 */
} lbem_ntff_desc;
int32_t lbem_far_field_noalloc(const lbem_ntff_desc *desc, const double *dft_dev,
                               const double *theta_dev, const double *phi_dev, int32_t n,
                               double *s2_dev, double *amp_dev, void *cuda_stream);

/* Wait for the handle's stream; reports an asynchronous CUDA error. */
int32_t lbem_sync(lbem_handle h);

void lbem_destroy(lbem_handle h);

/* Message of the last failed call on h (or of the last failed lbem_create when
 * h is NULL); never NULL. */
const char *lbem_last_error(lbem_handle h);

/* Kernel launches this handle has issued since creation (every lbem_* call
 * counts the kernels it enqueues). */
int64_t lbem_kernel_launches(lbem_handle h);

#ifdef __cplusplus
}
#endif

#endif /* LBEM_H */
