// Internal definitions shared by the CUDA translation units of liblbem.
// The public C ABI is include/lbem.h.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstddef>
#include <cstdint>

namespace lbem {

constexpr int kMaxDevices = 64;  // per-device set-up caches
// Buffers of the incident line: a two-step pass reads line(n+1) and line(n+2)
// while its first block may already advance the line for the next pass,
// reading line(n+3) and writing line(n+4) and line(n+5).
constexpr int kLineBufs = 5;
// Streaming multiprocessors and L2 bytes of the current device (queried once
// per device; 0 if the query fails).
int sm_count();
long long l2_bytes();

constexpr int kMaxQ = 42;        // 2 families x 7 directions x 3 components (3D)
constexpr int kMaxFaces = 6;
constexpr int kAngleBatch = 1024;  // angles per far-field kernel pass
constexpr int kMaxChunks = 128;    // face-cell chunks per angle in the projection

// Per-mode population planes (Sec. 2.1, D3Q7 with 3-vector populations).  A
// family stores only the vector components that are non-zero in the mode:
//   mode 0 (EZ): e_z ; h_x h_y     mode 1 (HZ): e_x e_y ; h_z     mode 2 (3D): all
// Plane q: e-planes q = i*NE + k, then h-planes q = 7*NE + i*NH + k.
template <int MODE> struct Mode;
template <> struct Mode<0> {
    static constexpr int NE = 1, NH = 2;
    __host__ __device__ static constexpr int ec(int) { return 2; }
    __host__ __device__ static constexpr int hc(int k) { return k; }
};
template <> struct Mode<1> {
    static constexpr int NE = 2, NH = 1;
    __host__ __device__ static constexpr int ec(int k) { return k; }
    __host__ __device__ static constexpr int hc(int) { return 2; }
};
template <> struct Mode<2> {
    static constexpr int NE = 3, NH = 3;
    __host__ __device__ static constexpr int ec(int k) { return k; }
    __host__ __device__ static constexpr int hc(int k) { return k; }
};
template <int MODE> struct Planes {
    using M = Mode<MODE>;
    static constexpr int NE = M::NE, NH = M::NH;
    static constexpr int Q = 7 * (NE + NH);
    static constexpr int NC = NE + NH;  // field components recorded by the DFT
    __host__ __device__ static constexpr int dir(int q) { return q < 7 * NE ? q / NE : (q - 7 * NE) / NH; }
    __host__ __device__ static constexpr int fam(int q) { return q < 7 * NE ? 0 : 1; }
    __host__ __device__ static constexpr int comp(int q) {
        return q < 7 * NE ? M::ec(q % NE) : M::hc((q - 7 * NE) % NH);
    }
};

inline int planes_of_mode(int mode) { return mode == 2 ? 42 : 21; }
inline int dft_comps_of_mode(int mode) { return mode == 2 ? 6 : 3; }

// ------------------------------------------------ population storage layout
// The populations of one buffer are grouped by direction.  Direction i holds
// the NC = NE + NH scalars of that direction in slots s = 0..NC-1 (the mode's
// e components, then its h components) in a block of NC*P elements starting
// at element i*NC*P (P: plane stride, cells padded in x).  The block is split
// into groups of consecutive slots; a group of width W whose first slot is s0
// starts at element (i*NC + s0)*P and keeps cell c's slot s at
// (i*NC + s0)*P + W*c + (s - s0), so one vector access fetches a whole group
// of a cell (all of a group's slots stream along the same velocity c_i):
//   3D FP32:  {e_x e_y} {e_z h_x} {h_y h_z}   three 8-byte pairs
//   3D 16-bit: {e_x e_y e_z h_x} {h_y h_z}    one 8-byte quad and one 4-byte pair
//   2D (both): {s0 s1} {s2}                   a pair and a single
// The buffer size is Q*P elements as for plain planes, and the start of plane
// slot q' = i*NC + s0 (q'*P elements) is where a group begins.
__host__ __device__ constexpr int mode_NE(int mode) { return mode == 0 ? 1 : (mode == 1 ? 2 : 3); }
__host__ __device__ constexpr int mode_NH(int mode) { return mode == 0 ? 2 : (mode == 1 ? 1 : 3); }
// population plane q (e-planes q = i*NE + k, then h-planes 7*NE + i*NH + k) -> direction / slot
__host__ __device__ constexpr int plane_dir(int mode, int q)
{
    return q < 7 * mode_NE(mode) ? q / mode_NE(mode) : (q - 7 * mode_NE(mode)) / mode_NH(mode);
}
__host__ __device__ constexpr int plane_slot(int mode, int q)
{
    return q < 7 * mode_NE(mode) ? q % mode_NE(mode)
                                 : mode_NE(mode) + (q - 7 * mode_NE(mode)) % mode_NH(mode);
}
__host__ __device__ constexpr int slot_plane(int mode, int i, int s)
{
    return s < mode_NE(mode) ? i * mode_NE(mode) + s
                             : 7 * mode_NE(mode) + i * mode_NH(mode) + (s - mode_NE(mode));
}
__host__ __device__ constexpr int group_first(int nc, int elem_bytes, int s)
{
    return nc == 3 ? (s < 2 ? 0 : 2) : (elem_bytes == 4 ? (s & ~1) : (s < 4 ? 0 : 4));
}
__host__ __device__ constexpr int group_width(int nc, int elem_bytes, int s)
{
    return nc == 3 ? (s < 2 ? 2 : 1) : (elem_bytes == 4 ? 2 : (s < 4 ? 4 : 2));
}
// Element index of plane q, cell c (c = z*ny*nxp + y*nxp + x).
__host__ __device__ inline long long pop_index(int mode, int elem_bytes, long long P, int q, long long c)
{
    const int nc = mode_NE(mode) + mode_NH(mode);
    const int i = plane_dir(mode, q), s = plane_slot(mode, q);
    const int s0 = group_first(nc, elem_bytes, s), w = group_width(nc, elem_bytes, s);
    return ((long long)i * nc + s0) * P + (long long)w * c + (s - s0);
}

// ------------------------------------------------ device helpers shared by
// the step, adjoint and observable kernels
// x/3 to within rounding: the constant 1/3 split into a float and a remainder,
// x*hi + x*lo evaluated with one rounding (FMA).  A plain x * fl(1/3) is biased
// upwards (fl(1/3) > 1/3), which would make the collision grow D and B by
// ~2e-8 per step; this form is unbiased.
constexpr float kThirdHi = 0.333333343267f;     // fl(1/3)
constexpr float kThirdLo = -9.934107481e-09f;   // 1/3 - fl(1/3)
__device__ __forceinline__ float third(float x) { return fmaf(x, kThirdHi, x * kThirdLo); }

// Direction i = 0..6: rest, +x, -x, +y, -y, +z, -z.
__host__ __device__ constexpr int dir_axis(int i) { return i == 0 ? -1 : (i - 1) / 2; }
__host__ __device__ constexpr int dir_sign(int i) { return i == 0 ? 0 : ((i & 1) ? 1 : -1); }

// (c_i x V)_a for an axis-aligned unit velocity c_i.
__device__ __forceinline__ float cross_c(int i, const float V[3], int a)
{
    const int d = dir_axis(i);
    const float s = (float)dir_sign(i);
    // e_x x V = (0, -Vz, Vy), e_y x V = (Vz, 0, -Vx), e_z x V = (-Vy, Vx, 0)
    if (d == 0) return a == 0 ? 0.f : (a == 1 ? -s * V[2] : s * V[1]);
    if (d == 1) return a == 0 ? s * V[2] : (a == 1 ? 0.f : -s * V[0]);
    return a == 0 ? -s * V[1] : (a == 1 ? s * V[0] : 0.f);
}

__device__ __forceinline__ float layer_keep(int d, int w, float sigma_max, float inv_w)
{
    if (d >= w) return 1.f;
    const float m = (float)(w - d) * inv_w;
    return 1.f - sigma_max * m * m * m;
}

__device__ __forceinline__ bool in_box(int x, int y, int z, const int lo[3], const int hi[3])
{
    return x >= lo[0] && x <= hi[0] && y >= lo[1] && y <= hi[1] && z >= lo[2] && z <= hi[2];
}

// DFT slot of field component c (0..2) in each mode, or -1 when the mode does
// not carry it: EZ (E_z, H_x, H_y), HZ (E_x, E_y, H_z), 3D (E_x..E_z, H_x..H_z).
__host__ __device__ constexpr int slot_E(int mode, int c)
{
    return mode == 0 ? (c == 2 ? 0 : -1) : (mode == 1 ? (c < 2 ? c : -1) : c);
}
__host__ __device__ constexpr int slot_H(int mode, int c)
{
    return mode == 0 ? (c < 2 ? 1 + c : -1) : (mode == 1 ? (c == 2 ? 2 : -1) : 3 + c);
}

// Closed-form incident plane wave (analytic TF/SF source):
//   tau = t - 3 k.(p - r0),  s = amp ramp(tau) sin(omega tau),  E = s pol, H = s kxp,
// ramp(tau) = (1 - cos(pi tau / t_ramp)) / 2 on 0 < tau < t_ramp (0 before, 1 after).
struct PlaneWaveA {
    double k[3], pol[3], kxp[3];
    double amp, omega, t_ramp;
    double r0[3];
};

__device__ __forceinline__ double pw_amplitude(const PlaneWaveA &w, double px, double py, double pz,
                                               double t)
{
    const double tau = t - 3.0 * (w.k[0] * (px - w.r0[0]) + w.k[1] * (py - w.r0[1]) +
                                  w.k[2] * (pz - w.r0[2]));
    double ramp = 1.0;
    if (tau <= 0.0) ramp = 0.0;
    else if (tau < w.t_ramp) ramp = 0.5 * (1.0 - cos(M_PI * tau / w.t_ramp));
    return w.amp * ramp * sin(w.omega * tau);
}

// Arguments of the fused step kernel (passed by value).
struct StepArgs {
    const void *fin_q[kMaxQ];  // start of each input population plane
    void *fout_q[kMaxQ];       // start of each output population plane
    const float *inv_eps;
    const float *inv_mu;       // 1/mu_r per cell (the magnetic-media kernel only)
    int nx, ny, nz, nxp;       // extent and padded row pitch (elements)
    long long P;               // plane stride in elements = nz*ny*nxp
    int nblk_x;                // blocks per row (set by the launcher)
    int rows_per_block;        // rows (y fastest, then z) per block (launcher)
    int nblk_main;             // blocks covering the lattice (set by the launcher)
    int *status;               // kernel error flags (bit 0: a bounded wait ran out)
    // absorbing layer
    int w;
    float sigma_max, inv_w;
    // TF/SF source: 1 = the incident line at time n+1 ([Q][n_line]; line_n is
    // used only to start a fresh line), 2 = the analytic plane wave pw at the
    // input state's time tn
    int tfsf;
    PlaneWaveA pw;
    long long tn;
    // analytic source in FP32 (kind 2): per-axis tables over the grid
    // coordinates, concatenated x, y, z: pw_ph[p] = exp(-j w 3 k_a (p - r0_a)),
    // pw_d[p] = 3 k_a (p - r0_a); pw_wt[s] = exp(j w t_s) and pw_t[s] = t_s for
    // t_0 = n (pulled cells) and t_1 = n + 1 (the cell itself)
    const float2 *pw_ph;
    const float *pw_d;
    float2 pw_wt[2];
    float pw_t[2];
    float pw_amp, pw_t_ramp;
    float pw_polf[3], pw_kxpf[3];  // polarisation p and k x p in FP32
    int tf_lo[3], tf_hi[3];
    int inc_axis;
    const float *line_n;
    const float *line_n1;
    int n_line;
    // DFT of the near fields on the NTFF box surface
    int dft_on;
    double dft_c, dft_s;
    double dft_scale;          // 2/(P T): incident line (FP32 units)
    double dft_scale_cells;    // 2/(P T) times the storage scale: lattice cells
    double dft_sc, dft_ss;     // dft_scale_cells times cos, sin of the step's phase
    float *xstage;             // 3D, non-NULL: staged face fields go here ([NC][xs_n]) for dft_flush_x
    long long xs_n;            // cells of all faces (one component of one staged step)
    long long xs_start[kMaxFaces];  // first staged cell of each face
    int nt_lo[3], nt_hi[3];
    double *dft;
    long long face_off[kMaxFaces];
    int face_nu[kMaxFaces], face_nv[kMaxFaces];
    // incident line update line(n+1) -> line(n+2) (first blocks of the launch)
    int line_on;
    float *line_out;
    int src_index;
    float src_E[3], src_H[3];  // hard-source fields at time n+2
    double *line_dft;          // [n_line][3][2]
    // reduced-precision storage: stored = population / scale (power of two)
    float scale, inv_scale;
    // forward replay for the adjoint: total-field D of the pulled populations
    // (scattered D plus the incident D inside the total-field box), NE planes
    // of P floats, written only by the recording kernel
    float *rec;
};

// One problem of a batched run (device copy; see lbem_batch_run).
struct BatchProblem {
    StepArgs a;                 // static arguments; per-step fields filled in the kernel
    const char *f_base[2];      // the two population buffers
    float *line[kLineBufs];     // incident line buffers, line(t) in line[t % kLineBufs]
    long long plane_bytes;
    long long t0, steps;        // time at the start of the run, steps to take
    int cur0;                   // buffer holding f*(t0)
    int T;                      // period in steps
    int nitems;                 // work items (row tiles) of this problem
    int item0;                  // first work item in the batch's list
    int has_wave;
    double amp, t_ramp;         // incident amplitude and ramp length (steps)
    float pol[3], kxp[3];       // p_hat and k_hat x p_hat
    long long dft_t0;           // first field time of the DFT window (< 1: none)
    int dft_periods;
    double scale;               // storage scale
};

struct BatchArgs {
    const BatchProblem *probs;
    int nprob;
    int nitems;
    int rows_per_item;          // rows of 128-cell tiles per work item
    long long max_steps;
    unsigned *bar_count;        // grid barrier: arrivals and generation
    unsigned *bar_gen;
    int *status;                // bit 1: a grid-barrier wait ran out
};

// Launchers (step.cu)
cudaError_t launch_batch(int mode, int storage, const BatchArgs &b, int grid, cudaStream_t s);
cudaError_t launch_barrier_selftest(const BatchArgs &b, cudaStream_t s);
int batch_max_blocks_per_sm(int mode, int storage);
cudaError_t launch_step(int mode, int storage, const StepArgs &a, cudaStream_t s);
// Two steps in one pass (any mode and storage; variant 0: plain update, 1:
// with the per-cell mu_r map; 2, the closed-form source, is refused and
// reported not worthwhile): s1 the first
// step's arguments (reads fin_q), s2 the second's (writes fout_q, which must
// not alias s1.fin_q); with the incident line on, a one-block launch before
// it updates the line for both steps (two launches in all).
// share: how many grids step concurrently beside each other (the lanes of a
// batched run), which the choice and the launch shape take into account.
// ahead (2D, incident line on): the arguments of the next pass's two steps,
// whose line work the first block does (line(n+4), line(n+5)); line_ready: the
// previous pass did this pass's line work, so the one-block launch is left out.
cudaError_t launch_step2(int mode, int storage, int variant, const StepArgs &s1, const StepArgs &s2,
                         cudaStream_t s, int share = 1, const StepArgs *ahead = nullptr, bool line_ready = false);
bool step2_worthwhile(int mode, int storage, int variant, int nx, int ny, int nz, int share = 1);

// In-place streaming on one population buffer (aa.cu).  Face buffers of
// direction i = 1..6 on axis (i - 1) / 2 ([NC][fplane[axis]] storage
// elements, face cell k: the other two coordinates, the lower one fastest):
// fi[i] holds P_i of the cells whose upstream neighbour x - c_i is outside,
// fo[i] P_i of the cells whose downstream neighbour x + c_i is outside; NULL
// along 1-cell axes.
struct AaArgs {
    void *fi[7];
    void *fo[7];
    long long fplane[3];
};
// One step: kind 0 (push) from the canonical state, reading fin_q (slot i)
// and writing through fout_q aimed at slot opp(i); kind 1 (in place) from the
// streamed state, reading through fin_q aimed at slot opp(i) and writing
// fout_q (slot i).  fin_q and fout_q address the same buffer.  variant as
// for launch_step2 (0 plain, 1 mu_r map, 2 closed-form source).
cudaError_t launch_aa_step(int mode, int storage, int variant, int kind, const StepArgs &a, const AaArgs &g,
                           cudaStream_t s);
// Fill fi from a canonical state (after any change to the state other than
// an in-place step).
cudaError_t launch_aa_fill(int mode, int storage, const void *buf, long long P, int nx, int ny, int nz, int nxp,
                           const AaArgs &g, cudaStream_t s);
// Turn the streamed state (after a push step) into the canonical one.
cudaError_t launch_aa_canonical(int mode, int storage, void *buf, long long P, int nx, int ny, int nz, int nxp,
                                const AaArgs &g, cudaStream_t s);
// The step kernel with a per-cell mu_r (a.inv_mu), Eq. 2's h_0 = (mu_r - 1) H
cudaError_t launch_step_mu(int mode, int storage, const StepArgs &a, cudaStream_t s);
// The step kernel with the analytic plane-wave source (a.tfsf == 2; reads a.inv_mu)
cudaError_t launch_step_analytic(int mode, int storage, const StepArgs &a, cudaStream_t s);
cudaError_t launch_fill(float *p, long long n, float v, cudaStream_t s);
cudaError_t launch_line_init(int mode, const StepArgs &a, cudaStream_t s);
// The step kernel with a.rec written (FP32 storage; forward replay of the adjoint)
cudaError_t launch_step_record(int mode, const StepArgs &a, cudaStream_t s);

// Where the stored populations hold the scattered part G = F - I (inside the
// total-field box), diagnostics add the incident line back.
struct IncView {
    int on;                    // 1: incident line, 2: analytic plane wave
    int tf_lo[3], tf_hi[3];
    int axis;
    const float *line;         // incident line at the state's time, [Q][n]
    int n;
    int mode;                  // analytic: population planes of this mode
    PlaneWaveA pw;
    double t;                  // analytic: the state's time
};

// Observables and data movement (observe.cu)
struct FaceGeom {
    int nfaces;
    int axis[kMaxFaces], side[kMaxFaces];
    int nu[kMaxFaces], nv[kMaxFaces];
    long long off[kMaxFaces];  // offset in doubles of face f in the DFT array
    long long cell_start[kMaxFaces + 1];  // prefix sum of nu*nv
    int lo[3], hi[3];
};

// Deferred DFT of NTFF faces: two banks of kXBank steps of staged fields
// [step][NC][n] (n the cells of all faces, face f from start[f]); one flush
// sums one bank: the faces each of its steps staged and the steps' phase
// coefficients.
constexpr int kXBank = 8;
constexpr int kXStage = 2 * kXBank;
struct DftFlushArgs {
    const float *stage;
    long long n;
    int nc, cnt, nfaces;
    double *dft;
    long long start[kMaxFaces + 1];
    long long plane[kMaxFaces];     // nu * nv of each face
    long long face_off[kMaxFaces];
    unsigned mask[kXBank];
    double sc[kXBank], ss[kXBank];
};
// blocks = 0: one thread per summed value; blocks > 0: that many blocks
// (grid-stride), small enough to sit beside a running step kernel.
cudaError_t launch_dft_flush_x(const DftFlushArgs &a, cudaStream_t s, int blocks);

struct FarFieldArgs {
    const double *dft;
    const double *line_dft;
    FaceGeom g;
    int mode;
    int n_ang;
    const double *theta, *phi;
    double k;
    double center[3];
    double pol[3];
    int center_i0, center_i1;  // incident-line nodes bracketing the centre
    double ei_fixed;           // > 0: |E_I| given (analytic source) instead of the line's DFT
    int chunks;
    double *partial;           // [n_ang][chunks][12]
    double *s2;                // [n_ang]
    double *amp;               // [n_ang][12]
    // 3D FP32 contraction (far_field_f32); x32 == nullptr selects the FP64 kernels
    float2 *x32;               // packed face phasors [face][nup][4][nvp], weights folded in
    float2 *tab32;             // phase tables [n0 + n1 + n2][n_ang_pad]
    long long x32_cap, tab32_cap;  // capacities in float2
    int n_ang_pad;             // n_ang rounded up to the angle tile
    int uc;                    // face rows per chunk
    int nup[kMaxFaces], nvp[kMaxFaces];  // padded rows / columns per face
    long long off32[kMaxFaces + 1];      // face offsets in x32 (float2)
    int chunk_start[kMaxFaces + 1];      // first chunk of each face
};
cudaError_t launch_far_field(const FarFieldArgs &a, cudaStream_t s, int *launches);
cudaError_t launch_far_field_partial(const FarFieldArgs &a, cudaStream_t s);

cudaError_t launch_inv_eps(const float *eps, float *inv_eps, int nx, int ny, int nz, int nxp,
                           int *bad_flag, cudaStream_t s);
cudaError_t launch_pack(int mode, int storage, const void *f, long long P, int q, float scale, float *out,
                        int nx, int ny, int nz, int nxp, const IncView &inc, cudaStream_t s);
cudaError_t launch_unpack(int mode, int storage, void *f, long long P, int q, float inv_scale,
                          const float *in, int nx, int ny, int nz, int nxp, const IncView &inc,
                          cudaStream_t s);
cudaError_t launch_add_incident(int mode, int storage, void *f, long long P, int Q, float scale,
                                int nx, int ny, int nz, int nxp, const IncView &inc, float sign,
                                cudaStream_t s);
cudaError_t launch_probe(int mode, int storage, const void *f, float scale, long long P, int ny, int nxp,
                         const int *xyz, int n, const IncView &inc, float *out, cudaStream_t s);
cudaError_t launch_fields(int mode, int storage, const void *f, const float *inv_eps, const float *inv_mu,
                          float scale, long long P, int nx, int ny, int nz, int nxp,
                          const IncView &inc, int comp, float *out, cudaStream_t s);
cudaError_t launch_energy(int mode, int storage, const void *f, const float *inv_eps, const float *inv_mu,
                          float scale, long long P, int nx, int ny, int nz, int nxp,
                          const IncView &inc, double *partial, int max_partial, double *out,
                          cudaStream_t s, int *launches);

// ---------------------------------------------------------------- adjoint
// One backward step of the discrete adjoint (adjoint.cu).  lin_q holds
// mu(t+1) = dJ/du(t+1), the objective's sensitivity to the pulled populations
// of the next step; the kernel writes mu(t) and adds this step's term of
// dJ/d(1/eps_r) to grad.  FP32 populations in the grouped layout of the
// forward state (lin_q[q'] / lout_q[q'] start plane slot q', as fin_q / fout_q
// do); FP64 gradient accumulator.
struct AdjointArgs {
    const float *lin_q[kMaxQ];
    float *lout_q[kMaxQ];
    const float *inv_eps;
    const float *rec;          // total-field D of step t's pulled state, NE planes of P
    double *grad;              // [P]
    int nx, ny, nz, nxp;
    long long P;
    int nblk_x;
    int w;
    float sigma_max, inv_w;
    // sensitivity of J to the DFT samples of step t (fields at time t)
    int dft_on;
    double dft_c, dft_s, dft_scale;
    int nt_lo[3], nt_hi[3];
    const double *G;           // dJ/dX per DFT entry, complex, in the DFT array layout
    long long face_off[kMaxFaces];
    int face_nu[kMaxFaces], face_nv[kMaxFaces];
};

// Sensitivity of J = sum_k w_k |S(theta_k, phi_k)|^2 to the DFT phasors.
struct AdjWeightArgs {
    FaceGeom g;
    int mode;
    int n_ang;
    const double *theta, *phi, *weights;
    const double *amp;         // [n_ang][12]: N and L of each angle (far_field_finalize)
    const double *line_dft;
    double k;
    double center[3];
    double pol[3];
    int center_i0, center_i1;
    double *gamma;             // [n_ang][12]: dJ/dN, dJ/dL (complex) of each angle
    double *G;                 // output, DFT layout
};

cudaError_t launch_adjoint_step(int mode, const AdjointArgs &a, cudaStream_t s);
cudaError_t launch_adjoint_weights(const AdjWeightArgs &a, cudaStream_t s, int *launches);
cudaError_t launch_adjoint_finalize(const double *grad, const float *inv_eps, int nx, int ny, int nz,
                                    int nxp, float *out, cudaStream_t s);

}  // namespace lbem
