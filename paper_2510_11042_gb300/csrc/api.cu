// C ABI of liblbem (declared in include/lbem.h): handle life cycle, argument
// checking, workspace layout, the step loop and the far-field call.
#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/lbem.h"
#include "lbem_internal.cuh"

using namespace lbem;

struct lbem_ctx {
    lbem_grid_desc g;
    int Q = 0, NC = 0;
    int nxp = 0;
    long long P = 0;          // plane stride (elements)
    long long ncell = 0;
    size_t elem = 4;          // bytes per stored population
    cudaStream_t stream = nullptr;
    int device = 0;
    // workspace
    char *ws = nullptr;
    size_t ws_bytes = 0;
    bool owns_ws = false;
    void *f[2] = {nullptr, nullptr};
    int cur = 0;
    float *inv_eps = nullptr;
    float *inv_mu = nullptr;    // 1/mu_r plane (1 where no map is set); read when mu_on or analytic
    float2 *pw_ph = nullptr;    // analytic source: per-axis phase factors, then 3 k_a (p - r0_a)
    float *pw_d = nullptr;
    bool mu_on = false;
    bool analytic = false;      // the plane wave is the closed-form source, not the line
    PlaneWaveA pw;
    float *line[kLineBufs] = {};  // incident line, line(t) in line[t mod kLineBufs]
    int n_line_max = 0;
    double *dft = nullptr;
    size_t dft_doubles_max = 0;
    double *line_dft = nullptr;
    double *scratch = nullptr;  // far-field partials / energy partials
    size_t scratch_doubles = 0;
    float2 *x32 = nullptr;      // 3D far field in FP32: packed faces, then phase tables
    float2 *tab32 = nullptr;
    size_t x32_cap = 0, tab32_cap = 0;
    bool ff_fp64 = false;       // LBEM_FAR_FIELD_FP64: 3D projection by the FP64 kernels
    int fuse = 2;               // steps per pass over the populations (lbem_set_step_fusion)
    // in-place streaming (LBEM_STREAM_IN_PLACE): f[0] only, the face buffers
    bool aa = false;
    int aa_phase = 0;           // 0: canonical state, 1: streamed (after a push step)
    bool aa_fi_valid = false;   // aa_g.fi holds the clamped values of the canonical state
    AaArgs aa_g;
    int share = 1;              // grids stepping beside this one (the lanes of a batched run)
    // deferred DFT of NTFF faces (see dft_flush_x_kernel): two banks of
    // kXBank staging slots; a full bank is summed on fstream while the steps
    // fill the other one
    float *xstage = nullptr;    // [2][kXBank][NC][xs_n]
    size_t xstage_floats = 0;
    long long xs_n = 0;         // cells of all faces (0: no staging)
    unsigned xs_xmask = 0;      // the x faces (staged by single steps)
    unsigned xs_allmask = 0;    // every face (staged by two-step passes)
    int xs_bank = 0;            // the bank being filled
    int xs_cnt = 0;             // its staged steps
    bool xs_wide = false;       // a step staged faces beyond x that the step stream has not summed
    unsigned xs_masks[kXBank];
    double xs_sc[kXBank], xs_ss[kXBank];
    cudaStream_t fstream = nullptr;           // side stream of the bank sums (3D)
    cudaEvent_t xs_filled[2] = {nullptr, nullptr};
    cudaEvent_t xs_summed[2] = {nullptr, nullptr};
    bool xs_inflight[2] = {false, false};     // a sum of the bank may still run on fstream
    int xs_last = -1;                         // bank of the last sum launched on fstream
    float *stage = nullptr;     // one FP32 plane of ncell values
    int *flag = nullptr;
    // time and source
    int64_t t = 0;
    bool has_wave = false;
    lbem_plane_wave wave;
    int T = 0;
    double omega = 0.0;
    int inc_axis = 0, n_line = 0, src_index = 0;
    FaceGeom faces;
    size_t dft_doubles = 0;
    int64_t dft_t0 = -1;
    int dft_periods = 0;
    float scale = 1.f, inv_scale = 1.f;  // stored population = population / scale
    int64_t launches = 0;
    // adjoint: checkpoints of lbem_forward_checkpointed and the backward buffers
    char *adj_ws = nullptr;
    size_t adj_bytes = 0;
    bool adj_owns = false;
    bool adj_valid = false;
    int64_t adj_steps = 0;
    int adj_K = 0;
    double adj_replay_ms = 0.0, adj_backward_ms = 0.0;  // of the last lbem_adjoint
    char err[512];
};

static thread_local char g_create_err[512] = "";

namespace lbem {
// Message of a failed call that has no handle (read by lbem_last_error(NULL)).
void set_noctx_error(const char *msg) { snprintf(g_create_err, sizeof g_create_err, "%s", msg); }
}

static int fail(lbem_ctx *h, int code, const char *fmt, ...)
{
    char *buf = h ? h->err : g_create_err;
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, 512, fmt, ap);
    va_end(ap);
    return code;
}

static int cuda_fail(lbem_ctx *h, cudaError_t e, const char *what)
{
    return fail(h, LBEM_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define CK(h, call)                                               \
    do {                                                          \
        cudaError_t e_ = (call);                                  \
        if (e_ != cudaSuccess) return cuda_fail((h), e_, #call);  \
    } while (0)

// Kernel status word: a step kernel that gave up on a bounded wait sets bit 0.
static int check_status(lbem_ctx *h)
{
    int st = 0;
    CK(h, cudaMemcpyAsync(&st, h->flag + 1, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    if (st & 1) return fail(h, LBEM_ERR_TIMEOUT, "a step kernel gave up waiting for its staged copies");
    return LBEM_OK;
}

// In-place streaming: bring the state to the canonical layout (after a push
// step it is the streamed one) before anything reads or writes populations.
static int aa_settle(lbem_ctx *h)
{
    if (!h->aa || h->aa_phase == 0) return LBEM_OK;
    CK(h, launch_aa_canonical(h->g.mode, h->g.storage, h->f[0], h->P, h->g.nx, h->g.ny, h->g.nz, h->nxp, h->aa_g,
                              h->stream));
    h->launches += 3;
    h->aa_phase = 0;
    h->aa_fi_valid = false;
    return LBEM_OK;
}

#define AA_SETTLE(h)                           \
    do {                                       \
        const int rc_ = aa_settle(h);          \
        if (rc_ != LBEM_OK) return rc_;        \
    } while (0)

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

struct Layout {
    size_t f0, f1, inv_eps, inv_mu, pw_tab, line[kLineBufs], dft, line_dft, scratch, ff32, stage, flag, total;
    size_t x32_cap, tab32_cap;  // float2 capacities of the 3D FP32 far field (0 in 2D)
    size_t xstage, xstage_floats;  // staged face DFT fields
    size_t aa_faces;               // in-place streaming: FI and FO of the six directions
    long long fplane[3];           // face cells of each axis (0 along 1-cell axes)
    int Q, nxp, n_line_max;
    long long P, ncell;
    size_t elem, dft_doubles_max, scratch_doubles;
};

static int check_grid(const lbem_grid_desc *g, char *why, size_t n)
{
    if (!g) return snprintf(why, n, "grid description is NULL"), 0;
    if (g->nx < 1 || g->ny < 1 || g->nz < 1)
        return snprintf(why, n, "grid extents must be >= 1 (got %d x %d x %d)", g->nx, g->ny, g->nz), 0;
    if (g->mode < 0 || g->mode > 2) return snprintf(why, n, "unknown mode %d", g->mode), 0;
    if (g->storage < 0 || g->storage > 2) return snprintf(why, n, "unknown storage %d", g->storage), 0;
    if (g->streaming != LBEM_STREAM_TWO_BUFFERS && g->streaming != LBEM_STREAM_IN_PLACE)
        return snprintf(why, n, "unknown streaming %d", g->streaming), 0;
    if (g->mode != 2 && g->nz != 1)
        return snprintf(why, n, "the 2D modes (EZ, HZ) need nz == 1"), 0;
    if (g->mode == 2 && g->nz < 2) return snprintf(why, n, "3D mode needs nz >= 2"), 0;
    const long long nxp = (g->nx + 31) / 32 * 32;
    const long long P = nxp * g->ny * (long long)g->nz;
    if (P >= (1LL << 31)) return snprintf(why, n, "grid too large (plane of %lld elements)", P), 0;
    const int minext = g->mode == 2 ? std::min(g->nx, std::min(g->ny, g->nz)) : std::min(g->nx, g->ny);
    if (g->absorber_width < 0 || 2 * g->absorber_width >= minext)
        return snprintf(why, n, "absorber_width %d does not fit the grid", g->absorber_width), 0;
    if (!(g->sigma_max <= 1.0) || std::isnan(g->sigma_max))
        return snprintf(why, n, "sigma_max must be <= 1"), 0;
    return 1;
}

static Layout make_layout(const lbem_grid_desc *g)
{
    Layout L;
    L.Q = planes_of_mode(g->mode);
    L.nxp = (g->nx + 31) / 32 * 32;
    L.P = (long long)L.nxp * g->ny * g->nz;
    L.ncell = (long long)g->nx * g->ny * g->nz;
    L.elem = g->storage == LBEM_F32 ? 4 : 2;
    L.n_line_max = std::max(g->nx, std::max(g->ny, g->nz));
    const int NC = dft_comps_of_mode(g->mode);
    // DFT capacity: the faces of the whole grid bound those of any NTFF box
    const long long fx = (long long)g->ny * g->nz, fy = (long long)g->nx * g->nz,
                    fz = (long long)g->nx * g->ny;
    L.dft_doubles_max = (size_t)(2 * (fx + fy + (g->nz > 1 ? fz : 0))) * NC * 2;
    // far-field partial sums; the energy monitor's block partials (capped at
    // this size by launch_energy) share the region
    L.scratch_doubles = (size_t)kAngleBatch * kMaxChunks * 12 + kAngleBatch * 16;
    size_t o = 0;
    auto take = [&](size_t bytes) { size_t at = o; o = align256(o + bytes); return at; };
    const bool aa = g->streaming == LBEM_STREAM_IN_PLACE;
    L.f0 = take((size_t)L.Q * L.P * L.elem);
    L.f1 = aa ? 0 : take((size_t)L.Q * L.P * L.elem);
    const long long n3[3] = {g->nx, g->ny, g->nz};
    size_t face_bytes = 0;
    for (int ax = 0; ax < 3; ++ax) {
        L.fplane[ax] = (aa && n3[ax] > 1) ? L.ncell / n3[ax] : 0;
        // FI and FO of both directions, each 256-byte aligned for vector access
        if (L.fplane[ax]) face_bytes += 4 * align256((size_t)L.fplane[ax] * NC * L.elem);
    }
    L.aa_faces = take(face_bytes);
    L.inv_eps = take((size_t)L.P * 4);
    L.inv_mu = take((size_t)L.P * 4);
    L.pw_tab = take((size_t)(g->nx + g->ny + g->nz) * 12);
    for (int k = 0; k < kLineBufs; ++k) L.line[k] = take((size_t)L.Q * L.n_line_max * 4);
    L.dft = take(L.dft_doubles_max * 8);
    L.line_dft = take((size_t)L.n_line_max * 6 * 8);
    L.scratch = take(L.scratch_doubles * 8);
    // 3D far field in FP32: faces padded to 16 rows x 64 columns (the NTFF box
    // lies in the grid, so its faces are bounded by the grid's) and phase
    // tables for a batch of angles
    L.x32_cap = L.tab32_cap = 0;
    if (g->mode == 2) {
        const long long n[3] = {g->nx, g->ny, g->nz};
        for (int ax = 0; ax < 3; ++ax) {
            const long long nu = n[ax == 2 ? 1 : 2], nv = n[ax == 0 ? 1 : 0];
            L.x32_cap += 2 * ((nu + 15) / 16 * 16) * 4 * ((nv + 63) / 64 * 64);
        }
        L.tab32_cap = (size_t)(g->nx + g->ny + g->nz) * kAngleBatch;
    }
    L.ff32 = take((L.x32_cap + L.tab32_cap) * 8);
    // two banks of kXBank steps of face fields; the faces of any NTFF box are bounded by
    // the grid's faces
    L.xstage_floats = g->mode == 2 ? (size_t)kXStage * NC * 2 *
                                         ((size_t)g->ny * g->nz + (size_t)g->nx * g->nz + (size_t)g->nx * g->ny)
                                   : 0;
    L.xstage = take(L.xstage_floats * 4);
    L.stage = take((size_t)L.ncell * 4);
    L.flag = take(256);
    L.total = o;
    return L;
}

// One power-of-two scale for all planes of reduced-precision storage.  The
// stored values are scattered fields; 2^-10 keeps populations up to +-64 below
// the FP16 maximum (65504) and leaves values down to ~6e-8 normal.  BF16 has
// the FP32 exponent range and needs no scaling.
static void default_scale(lbem_ctx *h)
{
    h->scale = h->g.storage == LBEM_F16 ? std::ldexp(1.0f, -10) : 1.0f;
    h->inv_scale = 1.0f / h->scale;
}

static double ramp(double t, double tr)
{
    if (t <= 0) return 0.0;
    if (t >= tr) return 1.0;
    return 0.5 * (1.0 - std::cos(M_PI * t / tr));
}

// Hard-source fields of the incident line at time t: E = E0 ramp(t) sin(w t) p, H = k x E.
static void source_fields(const lbem_ctx *h, int64_t t, float E[3], float H[3])
{
    const double *d = h->wave.dir, *p = h->wave.pol;
    const double kxp[3] = {d[1] * p[2] - d[2] * p[1], d[2] * p[0] - d[0] * p[2],
                           d[0] * p[1] - d[1] * p[0]};
    const double ph = 2.0 * M_PI * (double)(t % h->T) / (double)h->T;
    const double s = h->wave.amplitude * ramp((double)t, h->wave.ramp_periods * h->T) * std::sin(ph);
    for (int c = 0; c < 3; ++c) {
        E[c] = (float)(s * p[c]);
        H[c] = (float)(s * kxp[c]);
    }
}

static float *line_at(lbem_ctx *h, int64_t t) { return h->line[(int)(((t % kLineBufs) + kLineBufs) % kLineBufs)]; }

static IncView inc_view(lbem_ctx *h)
{
    IncView v;
    std::memset(&v, 0, sizeof v);
    if (!h->has_wave) return v;
    v.on = h->analytic ? 2 : 1;
    for (int k = 0; k < 3; ++k) {
        v.tf_lo[k] = h->wave.tfsf_lo[k];
        v.tf_hi[k] = h->wave.tfsf_hi[k];
    }
    v.mode = h->g.mode;
    v.pw = h->pw;
    v.t = (double)h->t;
    if (h->analytic) return v;
    v.axis = h->inc_axis;
    v.line = line_at(h, h->t);
    v.n = h->n_line;
    return v;
}

static void fill_common_args(lbem_ctx *h, StepArgs &a)
{
    std::memset(&a, 0, sizeof a);
    a.inv_eps = h->inv_eps;
    a.inv_mu = h->mu_on ? h->inv_mu : nullptr;
    a.nx = h->g.nx; a.ny = h->g.ny; a.nz = h->g.nz; a.nxp = h->nxp;
    a.P = h->P;
    a.w = h->g.absorber_width;
    a.sigma_max = (float)h->g.sigma_max;
    a.inv_w = a.w > 0 ? 1.0f / (float)a.w : 0.f;
    a.scale = h->scale;
    a.inv_scale = h->inv_scale;
    a.status = h->flag + 1;
    if (!h->has_wave) return;
    a.tfsf = h->analytic ? 2 : 1;
    a.line_on = h->analytic ? 0 : 1;
    a.pw = h->pw;
    if (h->analytic) {
        a.inv_mu = h->inv_mu;
        a.pw_ph = h->pw_ph;
        a.pw_d = h->pw_d;
        a.pw_amp = (float)h->pw.amp;
        a.pw_t_ramp = (float)h->pw.t_ramp;
        for (int c = 0; c < 3; ++c) {
            a.pw_polf[c] = (float)h->pw.pol[c];
            a.pw_kxpf[c] = (float)h->pw.kxp[c];
        }
    }
    for (int k = 0; k < 3; ++k) {
        a.tf_lo[k] = h->wave.tfsf_lo[k];
        a.tf_hi[k] = h->wave.tfsf_hi[k];
        a.nt_lo[k] = h->wave.ntff_lo[k];
        a.nt_hi[k] = h->wave.ntff_hi[k];
    }
    a.inc_axis = h->inc_axis;
    a.n_line = h->n_line;
    a.src_index = h->src_index;
    a.dft = h->dft;
    for (int f = 0; f < h->faces.nfaces; ++f) {
        a.face_off[f] = h->faces.off[f];
        a.face_nu[f] = h->faces.nu[f];
        a.face_nv[f] = h->faces.nv[f];
    }
    a.line_dft = h->line_dft;
}

extern "C" {

int32_t lbem_workspace_bytes(const lbem_grid_desc *grid, size_t *bytes_out)
{
    char why[256];
    if (!bytes_out) return fail(nullptr, LBEM_ERR_ARG, "bytes_out is NULL");
    if (!check_grid(grid, why, sizeof why)) return fail(nullptr, LBEM_ERR_ARG, "%s", why);
    *bytes_out = make_layout(grid).total;
    return LBEM_OK;
}

static int upload_inverse(lbem_ctx *h, const float *v, int on_device, float *target, const char *name);

static int upload_eps(lbem_ctx *h, const float *eps, int on_device)
{
    return upload_inverse(h, eps, on_device, h->inv_eps, "eps_r");
}

// Validate a per-cell map (finite, >= 1) and store its reciprocal in target.
static int upload_inverse(lbem_ctx *h, const float *eps, int on_device, float *target, const char *name)
{
    const float *src = eps;
    if (!on_device) {
        CK(h, cudaMemcpyAsync(h->stage, eps, (size_t)h->ncell * 4, cudaMemcpyHostToDevice, h->stream));
        src = h->stage;
    }
    // validate first, so that a rejected map leaves the handle unchanged
    CK(h, cudaMemsetAsync(h->flag, 0, sizeof(int), h->stream));
    CK(h, launch_inv_eps(src, nullptr, h->g.nx, h->g.ny, h->g.nz, h->nxp, h->flag, h->stream));
    h->launches += 1;
    int bad = 0;
    CK(h, cudaMemcpyAsync(&bad, h->flag, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    if (bad) return fail(h, LBEM_ERR_ARG, "%s must be finite and >= 1 in every cell", name);
    CK(h, launch_inv_eps(src, target, h->g.nx, h->g.ny, h->g.nz, h->nxp, h->flag, h->stream));
    h->launches += 1;
    return LBEM_OK;
}

int32_t lbem_create(const lbem_grid_desc *grid, int32_t velocity_set, const float *eps_r,
                    int32_t eps_on_device, void *cuda_stream, void *workspace,
                    size_t workspace_bytes, lbem_handle *out)
{
    char why[256];
    if (!out) return fail(nullptr, LBEM_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (velocity_set != LBEM_D3Q7) return fail(nullptr, LBEM_ERR_ARG, "only LBEM_D3Q7 is supported");
    if (!check_grid(grid, why, sizeof why)) return fail(nullptr, LBEM_ERR_ARG, "%s", why);
    if (!eps_r) return fail(nullptr, LBEM_ERR_ARG, "eps_r is NULL");
    if (workspace && ((uintptr_t)workspace & 255))
        return fail(nullptr, LBEM_ERR_ARG, "workspace must be 256-byte aligned");
    const Layout L = make_layout(grid);
    if (workspace && workspace_bytes < L.total)
        return fail(nullptr, LBEM_ERR_OOM, "workspace of %zu bytes is smaller than the %zu needed",
                    workspace_bytes, L.total);
    lbem_ctx *h = new (std::nothrow) lbem_ctx();
    if (!h) return fail(nullptr, LBEM_ERR_OOM, "host allocation failed");
    h->g = *grid;
    if (!(h->g.sigma_max > 0.0)) h->g.sigma_max = 0.3;
    h->Q = L.Q;
    h->NC = dft_comps_of_mode(grid->mode);
    h->nxp = L.nxp;
    h->P = L.P;
    h->ncell = L.ncell;
    h->elem = L.elem;
    h->stream = (cudaStream_t)cuda_stream;
    h->err[0] = 0;
    cudaGetDevice(&h->device);
    if (grid->mode == 2) {
        bool ok = cudaStreamCreateWithFlags(&h->fstream, cudaStreamNonBlocking) == cudaSuccess;
        for (int b = 0; b < 2 && ok; ++b)
            ok = cudaEventCreateWithFlags(&h->xs_filled[b], cudaEventDisableTiming) == cudaSuccess &&
                 cudaEventCreateWithFlags(&h->xs_summed[b], cudaEventDisableTiming) == cudaSuccess;
        if (!ok) {
            cudaGetLastError();
            lbem_destroy(h);
            return fail(nullptr, LBEM_ERR_CUDA, "creating the DFT side stream failed");
        }
    }
    if (workspace) {
        h->ws = (char *)workspace;
        h->ws_bytes = workspace_bytes;
    } else {
        cudaError_t e = cudaMalloc((void **)&h->ws, L.total);
        if (e != cudaSuccess) {
            cudaGetLastError();
            h->ws = nullptr;
            lbem_destroy(h);
            return fail(nullptr, LBEM_ERR_OOM, "cudaMalloc of %zu bytes failed: %s", L.total,
                        cudaGetErrorString(e));
        }
        h->owns_ws = true;
        h->ws_bytes = L.total;
    }
    h->aa = grid->streaming == LBEM_STREAM_IN_PLACE;
    h->f[0] = h->ws + L.f0;
    h->f[1] = h->aa ? nullptr : h->ws + L.f1;
    std::memset(&h->aa_g, 0, sizeof h->aa_g);
    if (h->aa) {
        // FI then FO, each direction i = 1..6 on its axis: NC face planes
        char *p = h->ws + L.aa_faces;
        for (int ax = 0; ax < 3; ++ax) h->aa_g.fplane[ax] = L.fplane[ax];
        for (int k = 0; k < 2; ++k)
            for (int i = 1; i < 7; ++i) {
                const long long plane = L.fplane[(i - 1) / 2];
                if (plane == 0) continue;
                (k == 0 ? h->aa_g.fi : h->aa_g.fo)[i] = p;
                p += align256((size_t)plane * h->NC * L.elem);
            }
    }
    h->inv_eps = (float *)(h->ws + L.inv_eps);
    h->inv_mu = (float *)(h->ws + L.inv_mu);
    h->pw_ph = (float2 *)(h->ws + L.pw_tab);
    h->pw_d = (float *)(h->pw_ph + (grid->nx + grid->ny + grid->nz));
    for (int k = 0; k < kLineBufs; ++k) h->line[k] = (float *)(h->ws + L.line[k]);
    h->n_line_max = L.n_line_max;
    h->dft = (double *)(h->ws + L.dft);
    h->dft_doubles_max = L.dft_doubles_max;
    h->line_dft = (double *)(h->ws + L.line_dft);
    h->scratch = (double *)(h->ws + L.scratch);
    h->scratch_doubles = L.scratch_doubles;
    h->xstage = (float *)(h->ws + L.xstage);
    h->xstage_floats = L.xstage_floats;
    h->x32_cap = L.x32_cap;
    h->tab32_cap = L.tab32_cap;
    h->x32 = L.x32_cap ? (float2 *)(h->ws + L.ff32) : nullptr;
    h->tab32 = L.x32_cap ? h->x32 + L.x32_cap : nullptr;
    h->stage = (float *)(h->ws + L.stage);
    h->flag = (int *)(h->ws + L.flag);
    default_scale(h);
    int rc = LBEM_OK;
    cudaError_t e = cudaMemsetAsync(h->flag, 0, 256, h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->f[0], 0, (size_t)L.Q * L.P * L.elem, h->stream);
    if (e == cudaSuccess && h->f[1]) e = cudaMemsetAsync(h->f[1], 0, (size_t)L.Q * L.P * L.elem, h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->inv_eps, 0, (size_t)L.P * 4, h->stream);
    if (e == cudaSuccess) e = launch_fill(h->inv_mu, L.P, 1.0f, h->stream);
    if (e != cudaSuccess) rc = cuda_fail(h, e, "cudaMemsetAsync");
    if (rc == LBEM_OK) rc = upload_eps(h, eps_r, eps_on_device);
    if (rc != LBEM_OK) {
        snprintf(g_create_err, sizeof g_create_err, "%s", h->err);
        lbem_destroy(h);
        return rc;
    }
    *out = h;
    return LBEM_OK;
}

int32_t lbem_set_permittivity(lbem_handle h, const float *eps_r, int32_t eps_on_device)
{
    if (!h) return fail(nullptr, LBEM_ERR_ARG, "NULL handle");
    if (!eps_r) return fail(h, LBEM_ERR_ARG, "eps_r is NULL");
    h->adj_valid = false;
    return upload_eps(h, eps_r, eps_on_device);
}

int32_t lbem_set_permeability(lbem_handle h, const float *mu_r, int32_t mu_on_device)
{
    if (!h) return fail(nullptr, LBEM_ERR_ARG, "NULL handle");
    h->adj_valid = false;
    if (!mu_r) {
        h->mu_on = false;
        CK(h, launch_fill(h->inv_mu, h->P, 1.0f, h->stream));
        return LBEM_OK;
    }
    const int rc = upload_inverse(h, mu_r, mu_on_device, h->inv_mu, "mu_r");
    if (rc == LBEM_OK) h->mu_on = true;
    return rc;
}

static int axis_of(const double d[3])
{
    int ax = -1;
    for (int a = 0; a < 3; ++a) {
        if (std::fabs(d[a]) > 1e-12) {
            if (ax >= 0) return -1;
            ax = a;
        }
    }
    if (ax < 0 || std::fabs(d[ax] - 1.0) > 1e-12) return -1;
    return ax;
}

static void build_faces(lbem_ctx *h)
{
    FaceGeom &F = h->faces;
    const int n3[3] = {h->g.nx, h->g.ny, h->g.nz};
    F.nfaces = 0;
    long long off = 0, cells = 0;
    for (int a = 0; a < 3; ++a) {
        F.lo[a] = h->wave.ntff_lo[a];
        F.hi[a] = h->wave.ntff_hi[a];
    }
    for (int ax = 0; ax < 3; ++ax) {
        if (n3[ax] <= 1) continue;
        const int ua = ax == 2 ? 1 : 2, va = ax == 0 ? 1 : 0;
        const int nu = F.hi[ua] - F.lo[ua] + 1, nv = F.hi[va] - F.lo[va] + 1;
        for (int side = 0; side < 2; ++side) {
            const int f = F.nfaces++;
            F.axis[f] = ax;
            F.side[f] = side;
            F.nu[f] = nu;
            F.nv[f] = nv;
            F.off[f] = off;
            F.cell_start[f] = cells;
            off += (long long)h->NC * 2 * nu * nv;
            cells += (long long)nu * nv;
        }
    }
    F.cell_start[F.nfaces] = cells;
    h->dft_doubles = (size_t)off;
    // staging in 3D only; faces 0 and 1 are the x faces when the grid has an x extent
    h->xs_n = (h->g.mode == 2 && F.nfaces > 0) ? (long long)cells : 0;
    if ((size_t)h->xs_n * h->NC * kXStage > h->xstage_floats) h->xs_n = 0;  // cannot happen: bounded by the grid
    // the bank sums index with 32 bits; past that the faces are summed in place
    if ((long long)h->xs_n * h->NC * kXBank > INT_MAX || h->dft_doubles > (size_t)INT_MAX) h->xs_n = 0;
    h->xs_xmask = (F.nfaces >= 2 && F.axis[0] == 0) ? 3u : 0u;
    h->xs_allmask = (1u << F.nfaces) - 1u;
    h->xs_bank = 0;
    h->xs_cnt = 0;
    h->xs_wide = false;
}

static int inject_analytic(lbem_ctx *h, const lbem_plane_wave *w);

int32_t lbem_inject_plane_wave(lbem_handle h, const lbem_plane_wave *w)
{
    if (!h) return fail(nullptr, LBEM_ERR_ARG, "NULL handle");
    if (!w) return fail(h, LBEM_ERR_ARG, "wave is NULL");
    if (w->source_kind == LBEM_SOURCE_ANALYTIC) return inject_analytic(h, w);
    if (w->source_kind != LBEM_SOURCE_LINE) return fail(h, LBEM_ERR_ARG, "unknown source_kind %d", w->source_kind);
    const int n3[3] = {h->g.nx, h->g.ny, h->g.nz};
    const int ax = axis_of(w->dir);
    if (ax < 0) return fail(h, LBEM_ERR_ARG, "dir must be +x, +y or +z");
    if (h->g.mode != 2 && ax == 2) return fail(h, LBEM_ERR_ARG, "2D modes need dir in the xy plane");
    double pn = 0, pd = 0;
    for (int a = 0; a < 3; ++a) {
        pn += w->pol[a] * w->pol[a];
        pd += w->pol[a] * w->dir[a];
    }
    if (std::fabs(pn - 1.0) > 1e-9 || std::fabs(pd) > 1e-9)
        return fail(h, LBEM_ERR_ARG, "pol must be a unit vector orthogonal to dir");
    if (h->g.mode == 0 && (std::fabs(w->pol[0]) > 1e-12 || std::fabs(w->pol[1]) > 1e-12))
        return fail(h, LBEM_ERR_ARG, "EZ mode needs pol along z");
    if (h->g.mode == 1 && std::fabs(w->pol[2]) > 1e-12)
        return fail(h, LBEM_ERR_ARG, "HZ mode needs pol in the xy plane");
    const double T = 3.0 * w->wavelength;
    if (!(w->wavelength > 0) || std::fabs(T - std::round(T)) > 1e-9 || std::round(T) < 2)
        return fail(h, LBEM_ERR_ARG, "3*wavelength must be an integer >= 2 (the period in steps)");
    if (!(w->amplitude > 0) || !std::isfinite(w->amplitude))
        return fail(h, LBEM_ERR_ARG, "amplitude must be positive");
    if (!(w->ramp_periods >= 0)) return fail(h, LBEM_ERR_ARG, "ramp_periods must be >= 0");
    const int W = h->g.absorber_width;
    for (int a = 0; a < 3; ++a) {
        if (n3[a] == 1) {
            if (w->tfsf_lo[a] || w->tfsf_hi[a] || w->ntff_lo[a] || w->ntff_hi[a])
                return fail(h, LBEM_ERR_ARG, "box bounds along a 1-cell axis must be 0");
            continue;
        }
        if (!(W <= w->ntff_lo[a] && w->ntff_lo[a] < w->tfsf_lo[a] && w->tfsf_lo[a] <= w->tfsf_hi[a] &&
              w->tfsf_hi[a] < w->ntff_hi[a] && w->ntff_hi[a] <= n3[a] - 1 - W))
            return fail(h, LBEM_ERR_ARG,
                        "axis %d: need W <= ntff_lo < tfsf_lo <= tfsf_hi < ntff_hi <= n-1-W", a);
    }
    int src = w->source_index < 0 ? W + 2 : w->source_index;
    if (src < 0 || src >= w->tfsf_lo[ax] - 1)
        return fail(h, LBEM_ERR_ARG, "source_index must lie upstream of the total-field box");
    if (h->has_wave) {
        // the stored state holds scattered parts inside the old box: make it total again
        AA_SETTLE(h);
        h->aa_fi_valid = false;
        CK(h, launch_add_incident(h->g.mode, h->g.storage, h->f[h->cur], h->P, h->Q, h->scale, h->g.nx, h->g.ny,
                                  h->g.nz, h->nxp, inc_view(h), 1.0f, h->stream));
        h->launches += 1;
        CK(h, cudaStreamSynchronize(h->stream));
    }
    h->adj_valid = false;
    h->wave = *w;
    h->wave.source_index = src;
    h->has_wave = true;
    h->analytic = false;
    std::memset(&h->pw, 0, sizeof h->pw);
    h->T = (int)std::lround(T);
    h->omega = 2.0 * M_PI / h->T;
    h->inc_axis = ax;
    h->n_line = n3[ax];
    h->src_index = src;
    build_faces(h);
    h->dft_t0 = -1;
    h->dft_periods = 0;
    for (int k = 0; k < 3; ++k)
        CK(h, cudaMemsetAsync(h->line[k], 0, (size_t)h->Q * h->n_line_max * 4, h->stream));
    CK(h, cudaMemsetAsync(h->line_dft, 0, (size_t)h->n_line_max * 6 * 8, h->stream));
    CK(h, cudaMemsetAsync(h->dft, 0, h->dft_doubles * 8, h->stream));
    // the line runs one step ahead: line(t) = 0, line(t+1) = one update of it
    StepArgs a;
    fill_common_args(h, a);
    a.line_n = line_at(h, h->t);
    a.line_out = line_at(h, h->t + 1);
    source_fields(h, h->t + 1, a.src_E, a.src_H);
    CK(h, launch_line_init(h->g.mode, a, h->stream));
    h->launches += 1;
    return LBEM_OK;
}

// The closed-form plane-wave source (see lbem_plane_wave).
static int inject_analytic(lbem_ctx *h, const lbem_plane_wave *w)
{
    const int n3[3] = {h->g.nx, h->g.ny, h->g.nz};
    double dn = 0, pn = 0, pd = 0;
    for (int a = 0; a < 3; ++a) {
        dn += w->dir[a] * w->dir[a];
        pn += w->pol[a] * w->pol[a];
        pd += w->pol[a] * w->dir[a];
    }
    if (std::fabs(dn - 1.0) > 1e-9 || std::fabs(pn - 1.0) > 1e-9 || std::fabs(pd) > 1e-9)
        return fail(h, LBEM_ERR_ARG, "dir and pol must be orthogonal unit vectors");
    if (h->g.mode != 2 && std::fabs(w->dir[2]) > 1e-12)
        return fail(h, LBEM_ERR_ARG, "2D modes need dir in the xy plane");
    if (h->g.mode == 0 && (std::fabs(w->pol[0]) > 1e-12 || std::fabs(w->pol[1]) > 1e-12))
        return fail(h, LBEM_ERR_ARG, "EZ mode needs pol along z");
    if (h->g.mode == 1 && std::fabs(w->pol[2]) > 1e-12)
        return fail(h, LBEM_ERR_ARG, "HZ mode needs pol in the xy plane");
    const double T = 3.0 * w->wavelength;
    if (!(w->wavelength > 0) || std::fabs(T - std::round(T)) > 1e-9 || std::round(T) < 2)
        return fail(h, LBEM_ERR_ARG, "3*wavelength must be an integer >= 2 (the period in steps)");
    if (!(w->amplitude > 0) || !std::isfinite(w->amplitude))
        return fail(h, LBEM_ERR_ARG, "amplitude must be positive");
    if (!(w->ramp_periods >= 0)) return fail(h, LBEM_ERR_ARG, "ramp_periods must be >= 0");
    bool ntff = false;
    for (int a = 0; a < 3; ++a) ntff = ntff || w->ntff_lo[a] || w->ntff_hi[a];
    const int W = h->g.absorber_width;
    for (int a = 0; a < 3; ++a) {
        if (w->tfsf_lo[a] > w->tfsf_hi[a]) return fail(h, LBEM_ERR_ARG, "axis %d: tfsf_lo > tfsf_hi", a);
        if (n3[a] == 1) {
            if (w->ntff_lo[a] || w->ntff_hi[a])
                return fail(h, LBEM_ERR_ARG, "NTFF bounds along a 1-cell axis must be 0");
            continue;
        }
        if (ntff && !(W <= w->ntff_lo[a] && w->ntff_lo[a] < w->tfsf_lo[a] && w->tfsf_hi[a] < w->ntff_hi[a] &&
                      w->ntff_hi[a] <= n3[a] - 1 - W))
            return fail(h, LBEM_ERR_ARG,
                        "axis %d: an NTFF box needs W <= ntff_lo < tfsf_lo <= tfsf_hi < ntff_hi <= n-1-W", a);
    }
    if (h->has_wave) {
        AA_SETTLE(h);
        h->aa_fi_valid = false;
        CK(h, launch_add_incident(h->g.mode, h->g.storage, h->f[h->cur], h->P, h->Q, h->scale, h->g.nx,
                                  h->g.ny, h->g.nz, h->nxp, inc_view(h), 1.0f, h->stream));
        h->launches += 1;
        CK(h, cudaStreamSynchronize(h->stream));
    }
    h->adj_valid = false;
    h->wave = *w;
    h->has_wave = true;
    h->analytic = true;
    h->T = (int)std::lround(T);
    h->omega = 2.0 * M_PI / h->T;
    h->inc_axis = 0;
    h->n_line = 1;
    h->src_index = 0;
    PlaneWaveA &p = h->pw;
    for (int a = 0; a < 3; ++a) {
        p.k[a] = w->dir[a];
        p.pol[a] = w->pol[a];
        p.r0[a] = w->origin[a];
    }
    p.kxp[0] = w->dir[1] * w->pol[2] - w->dir[2] * w->pol[1];
    p.kxp[1] = w->dir[2] * w->pol[0] - w->dir[0] * w->pol[2];
    p.kxp[2] = w->dir[0] * w->pol[1] - w->dir[1] * w->pol[0];
    p.amp = w->amplitude;
    p.omega = h->omega;
    p.t_ramp = w->ramp_periods * h->T;
    // per-axis tables of the step kernel (FP64 here, FP32 there)
    {
        const int ntab = n3[0] + n3[1] + n3[2];
        std::vector<float2> ph(ntab);
        std::vector<float> dd(ntab);
        int o = 0;
        for (int ax = 0; ax < 3; ++ax)
            for (int q = 0; q < n3[ax]; ++q, ++o) {
                const double d = 3.0 * p.k[ax] * ((double)q - p.r0[ax]);
                const double psi = std::fmod(h->omega * d, 2.0 * M_PI);
                ph[o] = make_float2((float)std::cos(psi), (float)-std::sin(psi));
                dd[o] = (float)d;
            }
        CK(h, cudaMemcpyAsync(h->pw_ph, ph.data(), ntab * sizeof(float2), cudaMemcpyHostToDevice, h->stream));
        CK(h, cudaMemcpyAsync(h->pw_d, dd.data(), ntab * sizeof(float), cudaMemcpyHostToDevice, h->stream));
        CK(h, cudaStreamSynchronize(h->stream));
    }
    if (ntff) {
        build_faces(h);
    } else {
        h->faces.nfaces = 0;
        h->xs_n = 0;
        h->faces.cell_start[0] = 0;
        h->dft_doubles = 0;
    }
    h->dft_t0 = -1;
    h->dft_periods = 0;
    if (h->dft_doubles) CK(h, cudaMemsetAsync(h->dft, 0, h->dft_doubles * 8, h->stream));
    // the stored state holds scattered parts inside the new box
    AA_SETTLE(h);
    h->aa_fi_valid = false;
    CK(h, launch_add_incident(h->g.mode, h->g.storage, h->f[h->cur], h->P, h->Q, h->scale, h->g.nx, h->g.ny,
                              h->g.nz, h->nxp, inc_view(h), -1.0f, h->stream));
    h->launches += 1;
    return LBEM_OK;
}

int32_t lbem_set_dft_window(lbem_handle h, int64_t t_start, int32_t n_periods)
{
    if (!h) return fail(nullptr, LBEM_ERR_ARG, "NULL handle");
    if (!h->has_wave) return fail(h, LBEM_ERR_STATE, "inject a plane wave first");
    if (n_periods < 1 || t_start < 1) return fail(h, LBEM_ERR_ARG, "need t_start >= 1 and n_periods >= 1");
    h->adj_valid = false;
    h->dft_t0 = t_start;
    h->dft_periods = n_periods;
    CK(h, cudaMemsetAsync(h->dft, 0, h->dft_doubles * 8, h->stream));
    CK(h, cudaMemsetAsync(h->line_dft, 0, (size_t)h->n_line_max * 6 * 8, h->stream));
    return LBEM_OK;
}

// Make the step stream wait for every bank sum launched on the side stream
// (they run in order there, so the last one covers them all).
static int join_sums(lbem_ctx *h)
{
    if (h->xs_last < 0) return LBEM_OK;
    const int b = h->xs_last;
    h->xs_last = -1;
    h->xs_inflight[0] = h->xs_inflight[1] = false;
    CK(h, cudaStreamWaitEvent(h->stream, h->xs_summed[b], 0));
    return LBEM_OK;
}

// Sum the bank being filled into the DFT accumulators (dft_flush_x_kernel) and
// fill the other bank next.  beside: on the side stream, after the steps that
// filled the bank and beside the steps that follow (a small grid that shares
// the SMs with them); else on the step stream after every earlier sum, with a
// full grid, leaving the DFT complete on the step stream.
static int flush_x_stage(lbem_ctx *h, bool beside)
{
    if (!beside) {
        const int rc = join_sums(h);
        if (rc != LBEM_OK) return rc;
    }
    const int b = h->xs_bank;
    if (h->xs_cnt > 0) {
        DftFlushArgs f;
        std::memset(&f, 0, sizeof f);
        f.stage = h->xstage + (size_t)b * kXBank * h->NC * h->xs_n;
        f.n = h->xs_n;
        f.nc = h->NC;
        f.cnt = h->xs_cnt;
        f.nfaces = h->faces.nfaces;
        f.dft = h->dft;
        for (int k = 0; k < h->faces.nfaces; ++k) {
            f.start[k] = h->faces.cell_start[k];
            f.plane[k] = (long long)h->faces.nu[k] * h->faces.nv[k];
            f.face_off[k] = h->faces.off[k];
        }
        f.start[h->faces.nfaces] = h->faces.cell_start[h->faces.nfaces];
        for (int s = 0; s < h->xs_cnt; ++s) {
            f.mask[s] = h->xs_masks[s];
            f.sc[s] = h->xs_sc[s];
            f.ss[s] = h->xs_ss[s];
        }
        h->xs_cnt = 0;
        if (beside) {
            CK(h, cudaEventRecord(h->xs_filled[b], h->stream));
            CK(h, cudaStreamWaitEvent(h->fstream, h->xs_filled[b], 0));
            cudaError_t e = launch_dft_flush_x(f, h->fstream, sm_count());
            if (e != cudaSuccess) return cuda_fail(h, e, "DFT bank sum launch");
            CK(h, cudaEventRecord(h->xs_summed[b], h->fstream));
            h->xs_inflight[b] = true;
            h->xs_last = b;
        } else {
            cudaError_t e = launch_dft_flush_x(f, h->stream, 0);
            if (e != cudaSuccess) return cuda_fail(h, e, "DFT bank sum launch");
        }
        h->launches += 1;
        h->xs_bank = b ^ 1;
        // the steps that fill the other bank start after its last sum read it
        if (h->xs_inflight[b ^ 1]) {
            h->xs_inflight[b ^ 1] = false;
            CK(h, cudaStreamWaitEvent(h->stream, h->xs_summed[b ^ 1], 0));
        }
    }
    if (!beside) h->xs_wide = false;
    return LBEM_OK;
}

// Per-step arguments of the step from time tn to tn+1 reading population
// buffer in and writing buffer out (a holds the common arguments).
static void step_args_at(lbem_ctx *h, StepArgs &a, int64_t tn, int in, int out)
{
    const int64_t t = tn + 1;  // time of the fields this step computes
    const size_t plane_bytes = (size_t)h->P * h->elem;
    for (int q = 0; q < h->Q; ++q) {
        a.fin_q[q] = (const char *)h->f[in] + q * plane_bytes;
        a.fout_q[q] = (char *)h->f[out] + q * plane_bytes;
    }
    a.dft_on = 0;
    if (h->has_wave) {
        if (!h->analytic) {
            a.line_n = line_at(h, tn);
            a.line_n1 = line_at(h, tn + 1);
            a.line_out = line_at(h, tn + 2);
            source_fields(h, tn + 2, a.src_E, a.src_H);
        }
        a.tn = tn;
        if (h->analytic)
            for (int k = 0; k < 2; ++k) {
                const int64_t ts = tn + k;
                const double ph = 2.0 * M_PI * (double)(ts % h->T) / (double)h->T;  // w t_s mod 2 pi
                a.pw_wt[k] = make_float2((float)std::cos(ph), (float)std::sin(ph));
                a.pw_t[k] = (float)ts;
            }
        a.dft_on = (h->faces.nfaces > 0 && h->dft_t0 >= 1 && t >= h->dft_t0 &&
                    t < h->dft_t0 + (int64_t)h->dft_periods * h->T);
        if (a.dft_on) {
            const double ph = 2.0 * M_PI * (double)(t % h->T) / (double)h->T;
            a.dft_c = std::cos(ph);
            a.dft_s = std::sin(ph);
            a.dft_scale = 2.0 / ((double)h->dft_periods * h->T);  // line (FP32, unscaled)
            a.dft_scale_cells = a.dft_scale * h->scale;            // lattice (storage units)
            a.dft_sc = a.dft_scale_cells * a.dft_c;
            a.dft_ss = a.dft_scale_cells * a.dft_s;
        }
    }
    a.xstage = nullptr;
}

// Claim the next staging slot for a step with the DFT on, staging the faces
// in mask.
static void stage_slot(lbem_ctx *h, StepArgs &a, unsigned mask)
{
    if (!a.dft_on || h->xs_n == 0 || mask == 0) return;
    a.xstage = h->xstage + ((size_t)h->xs_bank * kXBank + h->xs_cnt) * h->NC * h->xs_n;
    a.xs_n = h->xs_n;
    for (int f = 0; f < h->faces.nfaces; ++f) a.xs_start[f] = h->faces.cell_start[f];
    h->xs_masks[h->xs_cnt] = mask;
    h->xs_sc[h->xs_cnt] = a.dft_sc;
    h->xs_ss[h->xs_cnt] = a.dft_ss;
    h->xs_wide = h->xs_wide || (mask & ~h->xs_xmask) != 0;
    ++h->xs_cnt;
}

// In-place streaming: aim the push step's writes (kind 0, through fout_q) or
// the in-place step's reads (kind 1, through fin_q) of direction i at slot
// opp(i) of the single buffer.
static void aa_aim(lbem_ctx *h, StepArgs &a, int kind)
{
    const size_t plane_bytes = (size_t)h->P * h->elem;
    for (int i = 0; i < 7; ++i) {
        const int o = i == 0 ? 0 : ((i & 1) ? i + 1 : i - 1);
        for (int s = 0; s < h->NC; ++s) {
            char *p = (char *)h->f[0] + (size_t)(o * h->NC + s) * plane_bytes;
            if (kind == 0)
                a.fout_q[i * h->NC + s] = p;
            else
                a.fin_q[i * h->NC + s] = p;
        }
    }
}

// The kernel variant of the update: 0 plain, 1 with the mu_r map, 2 with the
// closed-form source.
static int step_variant(const lbem_ctx *h) { return h->analytic ? 2 : (h->mu_on ? 1 : 0); }

// Whether lbem_step takes two steps per pass: fusion on, on a grid whose
// blocks fill the GPU.
static bool two_step_passes(lbem_ctx *h)
{
    return h->fuse == 2 && !h->aa &&
           step2_worthwhile(h->g.mode, h->g.storage, step_variant(h), h->g.nx, h->g.ny, h->g.nz, h->share);
}

// The steps of lbem_step; on an error the step stream is still joined with
// the side stream's sums, so later work on it sees a consistent DFT.
static int step_loop(lbem_ctx *h, int64_t n)
{
    StepArgs a;
    fill_common_args(h, a);
    const bool pairs = two_step_passes(h);
    StepArgs a2, la[2];
    if (pairs) {
        fill_common_args(h, a2);
        fill_common_args(h, la[0]);
        fill_common_args(h, la[1]);
    }
    bool line_ready = false;  // the previous pass advanced the incident line for this one
    for (int64_t k = 0; k < n;) {
        if (pairs && n - k >= 2) {
            // two steps in one pass: level n from f[cur], level n+2 into f[cur ^ 1]
            if (h->xs_cnt + 2 > kXBank) {
                const int rc = flush_x_stage(h, true);
                if (rc != LBEM_OK) return rc;
            }
            step_args_at(h, a, h->t, h->cur, h->cur ^ 1);
            step_args_at(h, a2, h->t + 1, h->cur ^ 1, h->cur ^ 1);
            const int cnt0 = h->xs_cnt;
            stage_slot(h, a, h->xs_allmask);
            stage_slot(h, a2, h->xs_allmask);
            // a 2D pass that another pass of this call follows advances the
            // incident line for it (the line work of steps t+2 and t+3)
            const bool ahead = a.line_on && h->g.mode != 2 && n - k >= 4;
            if (ahead) {
                step_args_at(h, la[0], h->t + 2, h->cur, h->cur ^ 1);
                step_args_at(h, la[1], h->t + 3, h->cur ^ 1, h->cur ^ 1);
            }
            cudaError_t e = launch_step2(h->g.mode, h->g.storage, step_variant(h), a, a2, h->stream, h->share,
                                         ahead ? la : nullptr, line_ready);
            if (e != cudaSuccess) {
                h->xs_cnt = cnt0;   // the claimed slots hold nothing
                return cuda_fail(h, e, "two-step kernel launch");
            }
            h->launches += (a.line_on && !line_ready) ? 2 : 1;
            line_ready = ahead;
            h->cur ^= 1;
            h->t += 2;
            k += 2;
        } else {
            // a single step updates the faces it does not stage in place, so
            // terms staged for them by two-step passes go in first, on the
            // step stream
            if (h->xs_wide) {
                const int rc = flush_x_stage(h, false);
                if (rc != LBEM_OK) return rc;
            }
            line_ready = false;
            const int kind = h->aa_phase;  // in-place streaming: 0 push, 1 in place
            if (h->aa && kind == 0 && !h->aa_fi_valid) {
                CK(h, launch_aa_fill(h->g.mode, h->g.storage, h->f[0], h->P, h->g.nx, h->g.ny, h->g.nz, h->nxp,
                                     h->aa_g, h->stream));
                h->launches += 1;
                h->aa_fi_valid = true;
            }
            if (h->aa) {
                step_args_at(h, a, h->t, 0, 0);
                aa_aim(h, a, kind);
            } else {
                step_args_at(h, a, h->t, h->cur, h->cur ^ 1);
            }
            const int cnt0 = h->xs_cnt;
            stage_slot(h, a, h->xs_xmask);
            cudaError_t e = h->aa       ? launch_aa_step(h->g.mode, h->g.storage, step_variant(h), kind, a,
                                                         h->aa_g, h->stream)
                            : h->analytic ? launch_step_analytic(h->g.mode, h->g.storage, a, h->stream)
                            : h->mu_on    ? launch_step_mu(h->g.mode, h->g.storage, a, h->stream)
                                          : launch_step(h->g.mode, h->g.storage, a, h->stream);
            if (e != cudaSuccess) {
                h->xs_cnt = cnt0;
                return cuda_fail(h, e, "step kernel launch");
            }
            h->launches += 1;
            if (h->aa) {
                h->aa_phase ^= 1;
                h->aa_fi_valid = kind == 1;  // the in-place step rewrote them; a push step used them up
            } else {
                h->cur ^= 1;
            }
            h->t += 1;
            k += 1;
        }
        if (h->xs_cnt == kXBank) {
            const int rc = flush_x_stage(h, true);
            if (rc != LBEM_OK) return rc;
        }
    }
    return flush_x_stage(h, false);  // every call leaves the DFT complete on the step stream
}

int32_t lbem_step(lbem_handle h, int64_t n)
{
    if (!h) return fail(nullptr, LBEM_ERR_ARG, "NULL handle");
    if (n < 0) return fail(h, LBEM_ERR_ARG, "n must be >= 0");
    const int rc = step_loop(h, n);
    if (rc != LBEM_OK && h->xs_last >= 0) {
        cudaStreamWaitEvent(h->stream, h->xs_summed[h->xs_last], 0);
        h->xs_last = -1;
        h->xs_inflight[0] = h->xs_inflight[1] = false;
    }
    return rc;
}

int32_t lbem_set_step_fusion(lbem_handle h, int32_t steps_per_pass)
{
    if (!h) return fail(nullptr, LBEM_ERR_ARG, "NULL handle");
    if (steps_per_pass != 1 && steps_per_pass != 2)
        return fail(h, LBEM_ERR_ARG, "steps_per_pass must be 1 or 2");
    h->fuse = steps_per_pass;
    return LBEM_OK;
}

int32_t lbem_get_step_fusion(lbem_handle h, int32_t *steps_per_pass)
{
    if (!h || !steps_per_pass) return fail(h, LBEM_ERR_ARG, "NULL argument");
    *steps_per_pass = two_step_passes(h) ? 2 : 1;
    return LBEM_OK;
}

// ------------------------------------------------------------ batched runs
struct lbem_batch_ctx {
    std::vector<lbem_ctx *> hs;
    cudaStream_t stream = nullptr;
    char *ws = nullptr;
    bool owns_ws = false;
    BatchProblem *table = nullptr;   // device
    unsigned *bar = nullptr;         // device: count, generation
    int *status = nullptr;           // device
    int mode = 0, storage = 0;
    int tuned = 0, best_bps = 0, best_rpi = 1;
    int split = 0;                   // large grids stepped by plain launches, the rest persistent
    long long split_cells = 0;       // size from which a grid counts as large
    double best_ms = 0.0;
    int64_t launches = 0;
    cudaStream_t lanes[4] = {};      // streams of the large grids in a split schedule
    cudaEvent_t lane_ev[5] = {};     // lane joins and the fork from the batch stream
    char err[512];
};

static int bfail(lbem_batch_ctx *b, int code, const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(b ? b->err : g_create_err, 512, fmt, ap);
    va_end(ap);
    return code;
}

static size_t batch_bytes(int count)
{
    return align256((size_t)count * sizeof(BatchProblem)) + 256;
}

extern "C" int32_t lbem_batch_workspace_bytes(int32_t count, size_t *bytes_out)
{
    if (count < 1 || !bytes_out) return bfail(nullptr, LBEM_ERR_ARG, "need count >= 1 and bytes_out");
    *bytes_out = batch_bytes(count);
    return LBEM_OK;
}

extern "C" int32_t lbem_batch_create(const lbem_handle *handles, int32_t count, void *cuda_stream,
                                     void *workspace, size_t workspace_bytes, lbem_batch *out)
{
    if (!out) return bfail(nullptr, LBEM_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (!handles || count < 1) return bfail(nullptr, LBEM_ERR_ARG, "need at least one handle");
    int dev = 0;
    cudaGetDevice(&dev);
    for (int i = 0; i < count; ++i) {
        if (!handles[i]) return bfail(nullptr, LBEM_ERR_ARG, "handle %d is NULL", i);
        if (handles[i]->g.mode != handles[0]->g.mode || handles[i]->g.storage != handles[0]->g.storage)
            return bfail(nullptr, LBEM_ERR_ARG, "all handles of a batch need the same mode and storage");
        if (handles[i]->mu_on)
            return bfail(nullptr, LBEM_ERR_ARG, "batched runs support mu_r = 1 only");
        if (handles[i]->analytic)
            return bfail(nullptr, LBEM_ERR_ARG, "batched runs need the incident-line source");
        if (handles[i]->aa)
            return bfail(nullptr, LBEM_ERR_ARG, "batched runs need two population buffers (not in-place streaming)");
        if (handles[i]->device != dev) return bfail(nullptr, LBEM_ERR_ARG, "handle %d is on another device", i);
        for (int j = 0; j < i; ++j)
            if (handles[j] == handles[i]) return bfail(nullptr, LBEM_ERR_ARG, "handle %d repeated", i);
    }
    const size_t need = batch_bytes(count);
    if (workspace && ((uintptr_t)workspace & 255)) return bfail(nullptr, LBEM_ERR_ARG, "workspace must be 256-byte aligned");
    if (workspace && workspace_bytes < need)
        return bfail(nullptr, LBEM_ERR_OOM, "batch workspace of %zu bytes < %zu", workspace_bytes, need);
    lbem_batch_ctx *b = new (std::nothrow) lbem_batch_ctx();
    if (!b) return bfail(nullptr, LBEM_ERR_OOM, "host allocation failed");
    b->hs.assign(handles, handles + count);
    b->stream = (cudaStream_t)cuda_stream;
    b->mode = handles[0]->g.mode;
    b->storage = handles[0]->g.storage;
    if (workspace) {
        b->ws = (char *)workspace;
    } else {
        if (cudaMalloc((void **)&b->ws, need) != cudaSuccess) {
            cudaGetLastError();
            delete b;
            return bfail(nullptr, LBEM_ERR_OOM, "cudaMalloc of the batch workspace failed");
        }
        b->owns_ws = true;
    }
    for (int l = 0; l < 4; ++l)
        if (cudaStreamCreateWithFlags(&b->lanes[l], cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            lbem_batch_destroy(b);
            return bfail(nullptr, LBEM_ERR_CUDA, "stream creation failed");
        }
    for (int l = 0; l < 5; ++l)
        if (cudaEventCreateWithFlags(&b->lane_ev[l], cudaEventDisableTiming) != cudaSuccess) {
            cudaGetLastError();
            lbem_batch_destroy(b);
            return bfail(nullptr, LBEM_ERR_CUDA, "event creation failed");
        }
    b->table = (BatchProblem *)b->ws;
    b->bar = (unsigned *)(b->ws + align256((size_t)count * sizeof(BatchProblem)));
    b->status = (int *)(b->bar + 2);
    b->err[0] = 0;
    *out = b;
    return LBEM_OK;
}

// Run every problem of the batch min(left_i, chunk) steps in one cooperative launch.
// Advance the problems listed in group by min(left, chunk) steps in one
// persistent launch.
static int batch_chunk(lbem_batch_ctx *b, std::vector<int64_t> &left, int64_t chunk, int bps, int rpi,
                       cudaEvent_t ev0, cudaEvent_t ev1, const std::vector<int> &group)
{
    const int n = (int)group.size();
    std::vector<BatchProblem> tab(n);
    int items = 0;
    int64_t max_steps = 0;
    for (int gi = 0; gi < n; ++gi) {
        const int i = group[gi];
        lbem_ctx *h = b->hs[i];
        BatchProblem &P = tab[gi];
        std::memset(&P, 0, sizeof P);
        fill_common_args(h, P.a);
        P.a.nblk_x = (h->g.nx + 127) / 128;
        const int rows = h->g.ny * h->g.nz;
        P.nitems = P.a.nblk_x * ((rows + rpi - 1) / rpi);
        P.a.nblk_main = P.nitems;
        if (h->has_wave && (h->n_line + 127) / 128 > P.nitems)
            return bfail(b, LBEM_ERR_ARG, "problem %d is too small for %d rows per work item", i, rpi);
        P.item0 = items;
        items += P.nitems;
        P.f_base[0] = (const char *)h->f[0];
        P.f_base[1] = (const char *)h->f[1];
        for (int k = 0; k < kLineBufs; ++k) P.line[k] = h->line[k];
        P.plane_bytes = (long long)h->P * (long long)h->elem;
        P.t0 = h->t;
        P.steps = std::min<int64_t>(left[i], chunk);
        P.cur0 = h->cur;
        P.scale = h->scale;
        P.has_wave = h->has_wave ? 1 : 0;
        if (h->has_wave) {
            P.T = h->T;
            P.amp = h->wave.amplitude;
            P.t_ramp = h->wave.ramp_periods * h->T;
            const double *d = h->wave.dir, *p = h->wave.pol;
            const double kxp[3] = {d[1] * p[2] - d[2] * p[1], d[2] * p[0] - d[0] * p[2], d[0] * p[1] - d[1] * p[0]};
            for (int c = 0; c < 3; ++c) {
                P.pol[c] = (float)p[c];
                P.kxp[c] = (float)kxp[c];
            }
            P.dft_t0 = h->dft_t0;
            P.dft_periods = h->dft_periods;
        } else {
            P.T = 1;
        }
        max_steps = std::max<int64_t>(max_steps, P.steps);
    }
    if (max_steps == 0) return LBEM_OK;
    if (cudaMemcpyAsync(b->table, tab.data(), n * sizeof(BatchProblem), cudaMemcpyHostToDevice, b->stream) != cudaSuccess ||
        cudaMemsetAsync(b->bar, 0, 2 * sizeof(unsigned) + sizeof(int), b->stream) != cudaSuccess)
        return bfail(b, LBEM_ERR_CUDA, "batch table upload failed");
    BatchArgs a;
    a.probs = b->table;
    a.nprob = n;
    a.nitems = items;
    a.rows_per_item = rpi;
    a.max_steps = max_steps;
    a.bar_count = b->bar;
    a.bar_gen = b->bar + 1;
    a.status = b->status;
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->hs[0]->device);
    const int grid = std::max(1, std::min(bps * sms, items));
    if (ev0) cudaEventRecord(ev0, b->stream);
    cudaError_t e = launch_batch(b->mode, b->storage, a, grid, b->stream);
    if (ev1) cudaEventRecord(ev1, b->stream);
    if (e != cudaSuccess) return bfail(b, LBEM_ERR_CUDA, "batch launch: %s", cudaGetErrorString(e));
    b->launches += 1;
    for (int gi = 0; gi < n; ++gi) {
        const int i = group[gi];
        lbem_ctx *h = b->hs[i];
        const int64_t k = tab[gi].steps;
        h->t += k;
        h->cur ^= (int)(k & 1);
        left[i] -= k;
    }
    int st = 0;
    if (cudaMemcpyAsync(&st, b->status, sizeof(int), cudaMemcpyDeviceToHost, b->stream) != cudaSuccess ||
        cudaStreamSynchronize(b->stream) != cudaSuccess)
        return bfail(b, LBEM_ERR_CUDA, "batch run: %s", cudaGetErrorString(cudaGetLastError()));
    if (st & 2) return bfail(b, LBEM_ERR_TIMEOUT, "a grid-barrier wait of the batched kernel ran out");
    return LBEM_OK;
}

// Grids of at least this many cells fill the GPU with one plain launch per
// step; the persistent kernel's grid barrier and shared-memory arguments only
// pay off below it.
constexpr long long kSplitCells = 1LL << 19;

// Steps per turn when the large grids take turns on the lanes.
constexpr int64_t kLaneSteps = 64;

// The large grids advance by plain step launches, the others in one
// persistent launch after them; ev0 / ev1 (optional) bracket both.  The large
// grids run on up to four lane streams, problem j always on lane j mod 4 (so
// its own steps stay in order), issued in turns of kLaneSteps steps: grids too
// small to fill the GPU alone, and the tail of every launch, then overlap with
// the other lanes' work.  The lanes fork from and join back into the batch
// stream through events.
static int split_chunk(lbem_batch_ctx *b, std::vector<int64_t> &left, int64_t chunk, int bps, int rpi,
                       const std::vector<int> &small, const std::vector<int> &big, cudaEvent_t ev0,
                       cudaEvent_t ev1)
{
    if (ev0) cudaEventRecord(ev0, b->stream);
    const int L = std::min<int>(4, (int)big.size());
    if (L > 0) {
        if (cudaEventRecord(b->lane_ev[4], b->stream) != cudaSuccess)
            return bfail(b, LBEM_ERR_CUDA, "lane fork failed");
        for (int l = 0; l < L; ++l)
            if (cudaStreamWaitEvent(b->lanes[l], b->lane_ev[4], 0) != cudaSuccess)
                return bfail(b, LBEM_ERR_CUDA, "lane fork failed");
    }
    std::vector<int64_t> todo(big.size());
    for (size_t j = 0; j < big.size(); ++j) todo[j] = std::min<int64_t>(left[big[j]], chunk);
    for (bool more = true; more;) {
        more = false;
        for (size_t j = 0; j < big.size(); ++j) {
            if (todo[j] == 0) continue;
            const int i = big[j];
            lbem_ctx *h = b->hs[i];
            const int64_t k = std::min<int64_t>(todo[j], kLaneSteps);
            cudaStream_t own = h->stream;
            h->stream = b->lanes[j % L];
            h->share = L;   // L grids step beside each other on the lanes
            const int64_t l0 = h->launches;
            const int rc = lbem_step(h, k);
            h->stream = own;
            h->share = 1;
            if (rc != LBEM_OK) return bfail(b, rc, "step of problem %d: %s", i, h->err);
            b->launches += h->launches - l0;
            left[i] -= k;
            todo[j] -= k;
            more = more || todo[j] > 0;
        }
    }
    for (int l = 0; l < L; ++l)
        if (cudaEventRecord(b->lane_ev[l], b->lanes[l]) != cudaSuccess ||
            cudaStreamWaitEvent(b->stream, b->lane_ev[l], 0) != cudaSuccess)
            return bfail(b, LBEM_ERR_CUDA, "lane join failed");
    if (!small.empty()) {
        const int rc = batch_chunk(b, left, chunk, bps, rpi, nullptr, nullptr, small);
        if (rc != LBEM_OK) return rc;
    }
    if (ev1) cudaEventRecord(ev1, b->stream);
    if (cudaStreamSynchronize(b->stream) != cudaSuccess)
        return bfail(b, LBEM_ERR_CUDA, "batch run: %s", cudaGetErrorString(cudaGetLastError()));
    return LBEM_OK;
}

extern "C" int32_t lbem_batch_run(lbem_batch b, const int64_t *steps, int32_t autotune)
{
    if (!b) return bfail(nullptr, LBEM_ERR_ARG, "NULL batch");
    if (!steps) return bfail(b, LBEM_ERR_ARG, "steps is NULL");
    const int n = (int)b->hs.size();
    std::vector<int64_t> left(steps, steps + n);
    for (int i = 0; i < n; ++i)
        if (left[i] < 0) return bfail(b, LBEM_ERR_ARG, "steps[%d] < 0", i);
    for (lbem_ctx *h : b->hs)
        if (cudaStreamSynchronize(h->stream) != cudaSuccess) return bfail(b, LBEM_ERR_CUDA, "handle stream failed");
    const int max_bps = batch_max_blocks_per_sm(b->mode, b->storage);
    if (max_bps < 1) return bfail(b, LBEM_ERR_CUDA, "the batched kernel cannot be resident");
    std::vector<int> all(n);
    for (int i = 0; i < n; ++i) all[i] = i;
    auto partition = [&](long long cells, std::vector<int> &small, std::vector<int> &big) {
        small.clear();
        big.clear();
        for (int i = 0; i < n; ++i) (b->hs[i]->ncell >= cells ? big : small).push_back(i);
    };
    if (autotune == 1 && !b->tuned) {
        // time a few steps of each candidate; steps taken while tuning count
        cudaEvent_t e0, e1;
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        const int64_t trial = 8;
        double best = 1e300;
        const int bps_c[4] = {1, 2, max_bps / 2, max_bps};
        const int rpi_c[3] = {1, 2, 4};
        for (int ib = 0; ib < 4; ++ib) {
            const int bps = std::max(1, std::min(max_bps, bps_c[ib]));
            for (int ir = 0; ir < 3; ++ir) {
                int64_t active = 0;
                for (int64_t v : left) active = std::max(active, std::min<int64_t>(v, trial));
                if (active < trial) break;
                int rc = batch_chunk(b, left, trial, bps, rpi_c[ir], e0, e1, all);
                if (rc != LBEM_OK) {
                    cudaEventDestroy(e0);
                    cudaEventDestroy(e1);
                    return rc;
                }
                float ms = 0.f;
                cudaEventElapsedTime(&ms, e0, e1);
                if (ms / trial < best) {
                    best = ms / trial;
                    b->best_bps = bps;
                    b->best_rpi = rpi_c[ir];
                }
            }
        }
        // split schedules (plain launches for the grids of at least 2^k cells)
        // against the all-persistent one, over the same number of trial steps
        for (int lg = 20; lg >= 16 && b->best_bps > 0; --lg) {
            std::vector<int> small, big;
            partition(1LL << lg, small, big);
            if (big.empty()) continue;
            int64_t active = 0;
            for (int64_t v : left) active = std::max(active, std::min<int64_t>(v, trial));
            if (active < trial) break;
            int rc = split_chunk(b, left, trial, b->best_bps, b->best_rpi, small, big, e0, e1);
            if (rc != LBEM_OK) {
                cudaEventDestroy(e0);
                cudaEventDestroy(e1);
                return rc;
            }
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (ms / trial < best) {
                best = ms / trial;
                b->split = 1;
                b->split_cells = 1LL << lg;
            }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        if (b->best_bps > 0) {
            b->tuned = 1;
            b->best_ms = best;
        }
    }
    if (autotune == 2) {
        b->split = 1;
        b->split_cells = kSplitCells;
    }
    const int bps = b->best_bps > 0 ? b->best_bps : max_bps;
    std::vector<int> small, big;
    if (b->split) partition(b->split_cells, small, big);
    if (b->split && !big.empty()) {
        int64_t remaining = 0;
        for (int64_t v : left) remaining = std::max(remaining, v);
        return split_chunk(b, left, remaining, bps, b->best_rpi, small, big, nullptr, nullptr);
    }
    int64_t remaining = 0;
    for (int64_t v : left) remaining = std::max(remaining, v);
    return batch_chunk(b, left, remaining, bps, b->best_rpi, nullptr, nullptr, all);
}

extern "C" int32_t lbem_batch_config(lbem_batch b, int32_t *blocks_per_sm, int32_t *rows_per_item,
                                     double *ms_per_step, int32_t *split)
{
    if (!b) return bfail(nullptr, LBEM_ERR_ARG, "NULL batch");
    if (split) *split = b->split;
    if (blocks_per_sm) *blocks_per_sm = b->best_bps;
    if (rows_per_item) *rows_per_item = b->best_rpi;
    if (ms_per_step) *ms_per_step = b->best_ms;
    return LBEM_OK;
}

extern "C" int32_t lbem_batch_selftest_barrier(lbem_batch b)
{
    if (!b) return bfail(nullptr, LBEM_ERR_ARG, "NULL batch");
    if (cudaMemsetAsync(b->bar, 0, 2 * sizeof(unsigned) + sizeof(int), b->stream) != cudaSuccess)
        return bfail(b, LBEM_ERR_CUDA, "barrier reset failed");
    BatchArgs a;
    std::memset(&a, 0, sizeof a);
    a.bar_count = b->bar;
    a.bar_gen = b->bar + 1;
    a.status = b->status;
    if (launch_barrier_selftest(a, b->stream) != cudaSuccess)
        return bfail(b, LBEM_ERR_CUDA, "self-test launch: %s", cudaGetErrorString(cudaGetLastError()));
    b->launches += 1;
    int st = 0;
    if (cudaMemcpyAsync(&st, b->status, sizeof(int), cudaMemcpyDeviceToHost, b->stream) != cudaSuccess ||
        cudaStreamSynchronize(b->stream) != cudaSuccess)
        return bfail(b, LBEM_ERR_CUDA, "self-test: %s", cudaGetErrorString(cudaGetLastError()));
    if (st & 2) return bfail(b, LBEM_ERR_TIMEOUT, "a grid-barrier wait of the batched kernel ran out");
    return bfail(b, LBEM_ERR_STATE, "the barrier self-test's wait did not run out");
}

extern "C" int64_t lbem_batch_launches(lbem_batch b) { return b ? b->launches : 0; }

extern "C" const char *lbem_batch_last_error(lbem_batch b) { return b ? b->err : g_create_err; }

extern "C" void lbem_batch_destroy(lbem_batch b)
{
    if (!b) return;
    for (int l = 0; l < 4; ++l)
        if (b->lanes[l]) {
            cudaStreamSynchronize(b->lanes[l]);
            cudaStreamDestroy(b->lanes[l]);
        }
    for (int l = 0; l < 5; ++l)
        if (b->lane_ev[l]) cudaEventDestroy(b->lane_ev[l]);
    if (b->owns_ws) {
        cudaStreamSynchronize(b->stream);
        cudaFree(b->ws);
    }
    delete b;
}

int32_t lbem_get_time(lbem_handle h, int64_t *t_out)
{
    if (!h || !t_out) return fail(h, LBEM_ERR_ARG, "NULL argument");
    *t_out = h->t;
    return LBEM_OK;
}

// Chunks of the far-field projection per angle: enough blocks for the face
// cells (4096 per chunk) and for the face columns (256 per chunk).
static int far_field_chunks(const FaceGeom &g)
{
    const long long cells = g.cell_start[g.nfaces];
    long long cols = 0;
    for (int f = 0; f < g.nfaces; ++f) cols += g.nv[f];
    const long long c = std::max((cells + 4095) / 4096, (cols + 255) / 256);
    return (int)std::max<long long>(1, std::min<long long>(kMaxChunks, c));
}

// The 3D projection runs as an FP32 contraction in the workspace's ff32 region.
static void set_far_field_f32(lbem_ctx *h, FarFieldArgs &a)
{
    if (h->ff_fp64) return;  // x32 stays NULL: the FP64 kernels
    a.x32 = h->x32;
    a.tab32 = h->tab32;
    a.x32_cap = (long long)h->x32_cap;
    a.tab32_cap = (long long)h->tab32_cap;
}

static void centre_nodes(lbem_ctx *h, int *i0, int *i1)
{
    const double c = h->wave.center[h->inc_axis];
    int a = (int)std::floor(c);
    if (a < 0) a = 0;
    if (a > h->n_line - 1) a = h->n_line - 1;
    *i0 = a;
    *i1 = std::min(a + 1, h->n_line - 1);
}

int32_t lbem_far_field(lbem_handle h, const double *theta, const double *phi, int32_t n,
                       double *s2, double *amp)
{
    if (!h) return fail(nullptr, LBEM_ERR_ARG, "NULL handle");
    if (!h->has_wave) return fail(h, LBEM_ERR_STATE, "inject a plane wave first");
    if (n < 0 || (n > 0 && (!theta || !s2))) return fail(h, LBEM_ERR_ARG, "bad angle arrays");
    if (h->g.mode == 2 && n > 0 && !phi) return fail(h, LBEM_ERR_ARG, "3D needs phi");
    if (h->faces.nfaces == 0) return fail(h, LBEM_ERR_STATE, "the plane wave has no NTFF box");
    FarFieldArgs a;
    std::memset(&a, 0, sizeof a);
    a.ei_fixed = h->analytic ? h->wave.amplitude : 0.0;
    a.dft = h->dft;
    a.line_dft = h->line_dft;
    a.g = h->faces;
    a.mode = h->g.mode;
    a.k = 2.0 * M_PI / h->wave.wavelength;
    for (int c = 0; c < 3; ++c) {
        a.center[c] = h->wave.center[c];
        a.pol[c] = h->wave.pol[c];
    }
    centre_nodes(h, &a.center_i0, &a.center_i1);
    a.chunks = far_field_chunks(h->faces);
    double *d_theta = h->scratch;
    double *d_phi = d_theta + kAngleBatch;
    double *d_s2 = d_phi + kAngleBatch;
    double *d_amp = d_s2 + kAngleBatch;
    double *d_part = d_amp + (size_t)kAngleBatch * 12;
    for (int32_t b0 = 0; b0 < n; b0 += kAngleBatch) {
        const int nb = std::min<int32_t>(kAngleBatch, n - b0);
        CK(h, cudaMemcpyAsync(d_theta, theta + b0, nb * 8, cudaMemcpyHostToDevice, h->stream));
        if (h->g.mode == 2)
            CK(h, cudaMemcpyAsync(d_phi, phi + b0, nb * 8, cudaMemcpyHostToDevice, h->stream));
        a.theta = d_theta;
        a.phi = d_phi;
        a.n_ang = nb;
        a.partial = d_part;
        a.s2 = d_s2;
        a.amp = d_amp;
        set_far_field_f32(h, a);
        int l = 0;
        CK(h, launch_far_field(a, h->stream, &l));
        h->launches += l;
        CK(h, cudaMemcpyAsync(s2 + b0, d_s2, nb * 8, cudaMemcpyDeviceToHost, h->stream));
        if (amp)
            CK(h, cudaMemcpyAsync(amp + (size_t)b0 * 12, d_amp, (size_t)nb * 12 * 8,
                                  cudaMemcpyDeviceToHost, h->stream));
        CK(h, cudaStreamSynchronize(h->stream));
    }
    return LBEM_OK;
}

int32_t lbem_set_far_field_precision(lbem_handle h, int32_t precision)
{
    if (!h) return fail(nullptr, LBEM_ERR_ARG, "NULL handle");
    if (precision != LBEM_FAR_FIELD_MIXED && precision != LBEM_FAR_FIELD_FP64)
        return fail(h, LBEM_ERR_ARG, "precision must be LBEM_FAR_FIELD_MIXED (0) or LBEM_FAR_FIELD_FP64 (1)");
    h->ff_fp64 = precision == LBEM_FAR_FIELD_FP64;
    return LBEM_OK;
}

int32_t lbem_incident_amplitude(lbem_handle h, double *out)
{
    if (!h || !out) return fail(h, LBEM_ERR_ARG, "NULL argument");
    if (!h->has_wave) return fail(h, LBEM_ERR_STATE, "inject a plane wave first");
    if (h->analytic) {
        *out = h->wave.amplitude;
        return LBEM_OK;
    }
    int i0, i1;
    centre_nodes(h, &i0, &i1);
    double v[2][6];
    CK(h, cudaMemcpyAsync(v[0], h->line_dft + (size_t)i0 * 6, 48, cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaMemcpyAsync(v[1], h->line_dft + (size_t)i1 * 6, 48, cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    double ei = 0;
    for (int t = 0; t < 2; ++t) {
        double re = 0, im = 0;
        for (int c = 0; c < 3; ++c) {
            re += h->wave.pol[c] * v[t][2 * c];
            im += h->wave.pol[c] * v[t][2 * c + 1];
        }
        ei += 0.5 * std::sqrt(re * re + im * im);
    }
    *out = ei;
    return LBEM_OK;
}

int32_t lbem_get_populations(lbem_handle h, float *out, int32_t on_device)
{
    if (!h || !out) return fail(h, LBEM_ERR_ARG, "NULL argument");
    for (int q = 0; q < h->Q; ++q) {
        float *dst = on_device ? out + (size_t)q * h->ncell : h->stage;
        AA_SETTLE(h);
        CK(h, launch_pack(h->g.mode, h->g.storage, h->f[h->cur], h->P, q, h->scale, dst, h->g.nx, h->g.ny,
                          h->g.nz, h->nxp, inc_view(h), h->stream));
        h->launches += 1;
        if (!on_device)
            CK(h, cudaMemcpyAsync(out + (size_t)q * h->ncell, h->stage, (size_t)h->ncell * 4,
                                  cudaMemcpyDeviceToHost, h->stream));
    }
    CK(h, cudaStreamSynchronize(h->stream));
    return LBEM_OK;
}

int32_t lbem_set_populations(lbem_handle h, const float *in, int32_t on_device)
{
    if (!h || !in) return fail(h, LBEM_ERR_ARG, "NULL argument");
    h->adj_valid = false;
    for (int q = 0; q < h->Q; ++q) {
        const float *src = in + (size_t)q * h->ncell;
        if (!on_device) {
            CK(h, cudaMemcpyAsync(h->stage, src, (size_t)h->ncell * 4, cudaMemcpyHostToDevice, h->stream));
            src = h->stage;
        }
        AA_SETTLE(h);
        h->aa_fi_valid = false;
        CK(h, launch_unpack(h->g.mode, h->g.storage, h->f[h->cur], h->P, q, h->inv_scale, src, h->g.nx,
                            h->g.ny, h->g.nz, h->nxp, inc_view(h), h->stream));
        h->launches += 1;
        if (!on_device) CK(h, cudaStreamSynchronize(h->stream));  // stage is reused
    }
    return LBEM_OK;
}

int32_t lbem_probe(lbem_handle h, const int32_t *xyz, int32_t n, float *out)
{
    if (!h) return fail(nullptr, LBEM_ERR_ARG, "NULL handle");
    if (n < 0 || n > LBEM_PROBE_MAX || (n > 0 && (!xyz || !out)))
        return fail(h, LBEM_ERR_ARG, "need 0..%d cells with xyz and out", LBEM_PROBE_MAX);
    if (n == 0) return LBEM_OK;
    for (int k = 0; k < n; ++k)
        if (xyz[3 * k] < 0 || xyz[3 * k] >= h->g.nx || xyz[3 * k + 1] < 0 || xyz[3 * k + 1] >= h->g.ny ||
            xyz[3 * k + 2] < 0 || xyz[3 * k + 2] >= h->g.nz)
            return fail(h, LBEM_ERR_ARG, "probe cell %d (%d, %d, %d) is outside the grid", k, xyz[3 * k],
                        xyz[3 * k + 1], xyz[3 * k + 2]);
    // scratch: the cell list, then n * Q floats
    int *d_xyz = (int *)h->scratch;
    float *d_out = (float *)(h->scratch) + 3 * LBEM_PROBE_MAX;
    CK(h, cudaMemcpyAsync(d_xyz, xyz, (size_t)n * 3 * sizeof(int32_t), cudaMemcpyHostToDevice, h->stream));
    AA_SETTLE(h);
    CK(h, launch_probe(h->g.mode, h->g.storage, h->f[h->cur], h->scale, h->P, h->g.ny, h->nxp, d_xyz, n,
                       inc_view(h), d_out, h->stream));
    h->launches += 1;
    CK(h, cudaMemcpyAsync(out, d_out, (size_t)n * h->Q * sizeof(float), cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    return check_status(h);
}

int32_t lbem_fields(lbem_handle h, float *E, float *H, int32_t on_device)
{
    if (!h || !E || !H) return fail(h, LBEM_ERR_ARG, "NULL argument");
    for (int comp = 0; comp < 6; ++comp) {
        float *dst = (comp < 3 ? E : H) + (size_t)(comp % 3) * h->ncell;
        float *out = on_device ? dst : h->stage;
        AA_SETTLE(h);
        CK(h, launch_fields(h->g.mode, h->g.storage, h->f[h->cur], h->inv_eps, h->mu_on ? h->inv_mu : nullptr, h->scale, h->P,
                            h->g.nx, h->g.ny, h->g.nz, h->nxp, inc_view(h), comp, out, h->stream));
        h->launches += 1;
        if (!on_device) {
            CK(h, cudaMemcpyAsync(dst, h->stage, (size_t)h->ncell * 4, cudaMemcpyDeviceToHost, h->stream));
            CK(h, cudaStreamSynchronize(h->stream));
        }
    }
    CK(h, cudaStreamSynchronize(h->stream));
    return LBEM_OK;
}

int32_t lbem_dft_doubles(lbem_handle h, size_t *count)
{
    if (!h || !count) return fail(h, LBEM_ERR_ARG, "NULL argument");
    if (!h->has_wave) return fail(h, LBEM_ERR_STATE, "inject a plane wave first");
    *count = h->dft_doubles;
    return LBEM_OK;
}

int32_t lbem_get_dft(lbem_handle h, double *out)
{
    if (!h || !out) return fail(h, LBEM_ERR_ARG, "NULL argument");
    if (!h->has_wave) return fail(h, LBEM_ERR_STATE, "inject a plane wave first");
    CK(h, cudaMemcpyAsync(out, h->dft, h->dft_doubles * 8, cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    return LBEM_OK;
}

int32_t lbem_energy(lbem_handle h, double *out)
{
    if (!h || !out) return fail(h, LBEM_ERR_ARG, "NULL argument");
    double *d_out = h->scratch;
    double *part = h->scratch + 8;
    int l = 0;
    AA_SETTLE(h);
    CK(h, launch_energy(h->g.mode, h->g.storage, h->f[h->cur], h->inv_eps, h->mu_on ? h->inv_mu : nullptr, h->scale, h->P, h->g.nx,
                        h->g.ny, h->g.nz, h->nxp, inc_view(h), part, (int)(h->scratch_doubles - 8),
                        d_out, h->stream, &l));
    h->launches += l;
    CK(h, cudaMemcpyAsync(out, d_out, 8, cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    if (!std::isfinite(*out)) return fail(h, LBEM_ERR_NONFINITE, "non-finite population in the state");
    return check_status(h);
}

// checkpoint: header | populations | incident line | line DFT | face DFT
struct StateHeader {
    char magic[8];
    int32_t nx, ny, nz, mode, storage, Q;
    int64_t t;
    int64_t pop_bytes, line_bytes, line_dft_bytes, dft_bytes;
    float scale;            // storage scale the populations are stored with
    int32_t pad;
};

int32_t lbem_state_bytes(lbem_handle h, size_t *bytes)
{
    if (!h || !bytes) return fail(h, LBEM_ERR_ARG, "NULL argument");
    *bytes = sizeof(StateHeader) + (size_t)h->Q * h->P * h->elem + 2 * (size_t)h->Q * h->n_line_max * 4 +
             (size_t)h->n_line_max * 48 + h->dft_doubles_max * 8;
    return LBEM_OK;
}

int32_t lbem_save_state(lbem_handle h, void *buf, size_t bytes)
{
    size_t need = 0;
    if (!h || !buf) return fail(h, LBEM_ERR_ARG, "NULL argument");
    lbem_state_bytes(h, &need);
    if (bytes < need) return fail(h, LBEM_ERR_ARG, "buffer of %zu bytes < %zu", bytes, need);
    StateHeader hd;
    std::memset(&hd, 0, sizeof hd);
    std::memcpy(hd.magic, "LBEMSTA2", 8);
    hd.scale = h->scale;
    hd.nx = h->g.nx; hd.ny = h->g.ny; hd.nz = h->g.nz; hd.mode = h->g.mode; hd.storage = h->g.storage;
    hd.Q = h->Q;
    hd.t = h->t;
    hd.pop_bytes = (int64_t)h->Q * h->P * h->elem;
    hd.line_bytes = (int64_t)h->Q * h->n_line_max * 4;
    hd.line_dft_bytes = (int64_t)h->n_line_max * 48;
    hd.dft_bytes = (int64_t)h->dft_doubles_max * 8;
    char *p = (char *)buf;
    std::memcpy(p, &hd, sizeof hd);
    p += sizeof hd;
    AA_SETTLE(h);
    CK(h, cudaMemcpyAsync(p, h->f[h->cur], hd.pop_bytes, cudaMemcpyDeviceToHost, h->stream));
    p += hd.pop_bytes;
    for (int k = 0; k < 2; ++k) {  // incident line at t and t+1
        CK(h, cudaMemcpyAsync(p, line_at(h, h->t + k), hd.line_bytes, cudaMemcpyDeviceToHost, h->stream));
        p += hd.line_bytes;
    }
    CK(h, cudaMemcpyAsync(p, h->line_dft, hd.line_dft_bytes, cudaMemcpyDeviceToHost, h->stream));
    p += hd.line_dft_bytes;
    CK(h, cudaMemcpyAsync(p, h->dft, hd.dft_bytes, cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    return LBEM_OK;
}

int32_t lbem_load_state(lbem_handle h, const void *buf, size_t bytes)
{
    size_t need = 0;
    if (!h || !buf) return fail(h, LBEM_ERR_ARG, "NULL argument");
    lbem_state_bytes(h, &need);
    if (bytes < need) return fail(h, LBEM_ERR_ARG, "buffer of %zu bytes < %zu", bytes, need);
    StateHeader hd;
    std::memcpy(&hd, buf, sizeof hd);
    if (std::memcmp(hd.magic, "LBEMSTA2", 8) || hd.nx != h->g.nx || hd.ny != h->g.ny || hd.nz != h->g.nz ||
        hd.mode != h->g.mode || hd.storage != h->g.storage || hd.Q != h->Q)
        return fail(h, LBEM_ERR_ARG, "snapshot does not match this grid");
    h->adj_valid = false;
    const char *p = (const char *)buf + sizeof hd;
    if (h->aa) {  // the snapshot replaces the whole state, in the canonical layout
        h->aa_phase = 0;
        h->aa_fi_valid = false;
    }
    CK(h, cudaMemcpyAsync(h->f[h->cur], p, hd.pop_bytes, cudaMemcpyHostToDevice, h->stream));
    p += hd.pop_bytes;
    for (int k = 0; k < 2; ++k) {  // incident line at t and t+1 of the snapshot
        CK(h, cudaMemcpyAsync(line_at(h, hd.t + k), p, hd.line_bytes, cudaMemcpyHostToDevice,
                              h->stream));
        p += hd.line_bytes;
    }
    CK(h, cudaMemcpyAsync(h->line_dft, p, hd.line_dft_bytes, cudaMemcpyHostToDevice, h->stream));
    p += hd.line_dft_bytes;
    CK(h, cudaMemcpyAsync(h->dft, p, hd.dft_bytes, cudaMemcpyHostToDevice, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    h->t = hd.t;
    h->scale = hd.scale;
    h->inv_scale = 1.0f / hd.scale;
    return LBEM_OK;
}

int32_t lbem_set_storage_scale(lbem_handle h, float scale)
{
    if (!h) return fail(nullptr, LBEM_ERR_ARG, "NULL handle");
    int e;
    if (!(scale > 0) || !std::isfinite(scale) || std::frexp(scale, &e) != 0.5f)
        return fail(h, LBEM_ERR_ARG, "scale must be a positive power of two");
    if (h->g.storage == LBEM_F32) return LBEM_OK;
    // rescale the stored state so that it keeps its value
    const float ratio = h->scale / scale;
    if (ratio != 1.0f) {
        IncView none;
        std::memset(&none, 0, sizeof none);
        for (int q = 0; q < h->Q; ++q) {
            AA_SETTLE(h);
            CK(h, launch_pack(h->g.mode, h->g.storage, h->f[h->cur], h->P, q, ratio, h->stage, h->g.nx, h->g.ny,
                              h->g.nz, h->nxp, none, h->stream));
            AA_SETTLE(h);
            h->aa_fi_valid = false;
            CK(h, launch_unpack(h->g.mode, h->g.storage, h->f[h->cur], h->P, q, 1.0f, h->stage, h->g.nx, h->g.ny,
                                h->g.nz, h->nxp, none, h->stream));
            h->launches += 2;
        }
    }
    h->scale = scale;
    h->inv_scale = 1.0f / scale;
    return LBEM_OK;
}

int32_t lbem_get_storage_scale(lbem_handle h, float *scale)
{
    if (!h || !scale) return fail(h, LBEM_ERR_ARG, "NULL argument");
    *scale = h->scale;
    return LBEM_OK;
}

int32_t lbem_sync(lbem_handle h)
{
    if (!h) return fail(nullptr, LBEM_ERR_ARG, "NULL handle");
    CK(h, cudaStreamSynchronize(h->stream));
    CK(h, cudaGetLastError());
    return check_status(h);
}

void lbem_destroy(lbem_handle h)
{
    if (!h) return;
    if (h->fstream) cudaStreamSynchronize(h->fstream);
    if ((h->owns_ws && h->ws) || (h->adj_owns && h->adj_ws)) cudaStreamSynchronize(h->stream);
    for (int b = 0; b < 2; ++b) {
        if (h->xs_filled[b]) cudaEventDestroy(h->xs_filled[b]);
        if (h->xs_summed[b]) cudaEventDestroy(h->xs_summed[b]);
    }
    if (h->fstream) cudaStreamDestroy(h->fstream);
    if (h->owns_ws && h->ws) cudaFree(h->ws);
    if (h->adj_owns && h->adj_ws) cudaFree(h->adj_ws);
    delete h;
}

// ------------------------------------------------------------ adjoint
// Workspace of lbem_forward_checkpointed / lbem_adjoint:
//   checkpoints  one per segment of K steps: populations and the three incident-line buffers
//   replay       two population buffers and three line buffers for the forward replay
//   mu           two adjoint population buffers
//   rec          total-field D of every step of one segment (K x NE planes)
//   G            dJ/dX per DFT entry (DFT array layout)
//   grad         FP64 accumulator of dJ/d(1/eps_r), one per padded cell
//   gamma, wts   per-angle sensitivities and weights
struct AdjLayout {
    size_t ck0, ck_stride, ck_lines, rf[2], rline[3], mu[2], rec, G, grad, gamma, wts, total;
    int nseg;
};

static AdjLayout adj_layout(const lbem_ctx *h, int64_t n_steps, int K)
{
    AdjLayout L;
    const size_t pop = (size_t)h->Q * h->P * 4;
    const size_t line = (size_t)h->Q * h->n_line_max * 4;
    const int NE = h->g.mode == 0 ? 1 : (h->g.mode == 1 ? 2 : 3);
    L.nseg = (int)((n_steps + K - 1) / K);
    L.ck_lines = align256(pop);
    L.ck_stride = L.ck_lines + 3 * align256(line);
    size_t o = 0;
    auto take = [&](size_t bytes) { size_t at = o; o = align256(o + bytes); return at; };
    L.ck0 = take(L.ck_stride * (size_t)L.nseg);
    for (int k = 0; k < 2; ++k) L.rf[k] = take(pop);
    for (int k = 0; k < 3; ++k) L.rline[k] = take(line);
    for (int k = 0; k < 2; ++k) L.mu[k] = take(pop);
    L.rec = take((size_t)K * NE * h->P * 4);
    L.G = take(h->dft_doubles_max * 8);
    L.grad = take((size_t)h->P * 8);
    L.gamma = take((size_t)kAngleBatch * 12 * 8);
    L.wts = take((size_t)kAngleBatch * 8);
    L.total = o;
    return L;
}

int32_t lbem_adjoint_workspace_bytes(lbem_handle h, int64_t n_steps, int32_t K, size_t *bytes)
{
    if (!h || !bytes) return fail(h, LBEM_ERR_ARG, "NULL argument");
    if (n_steps < 1 || K < 1) return fail(h, LBEM_ERR_ARG, "need n_steps >= 1 and K >= 1");
    *bytes = adj_layout(h, n_steps, K).total;
    return LBEM_OK;
}

int32_t lbem_forward_checkpointed(lbem_handle h, int64_t n_steps, int32_t K, void *workspace,
                                  size_t workspace_bytes)
{
    if (!h) return fail(nullptr, LBEM_ERR_ARG, "NULL handle");
    if (n_steps < 1 || K < 1) return fail(h, LBEM_ERR_ARG, "need n_steps >= 1 and K >= 1");
    if (h->g.storage != LBEM_F32) return fail(h, LBEM_ERR_ARG, "the adjoint needs FP32 storage");
    if (h->mu_on) return fail(h, LBEM_ERR_ARG, "the adjoint supports mu_r = 1 only");
    if (h->analytic) return fail(h, LBEM_ERR_ARG, "the adjoint needs the incident-line source");
    if (h->aa) return fail(h, LBEM_ERR_ARG, "the adjoint needs two population buffers (not in-place streaming)");
    if (!h->has_wave) return fail(h, LBEM_ERR_STATE, "inject a plane wave first");
    if (h->t != 0) return fail(h, LBEM_ERR_STATE, "the checkpointed run must start at t = 0 (got t = %lld)",
                               (long long)h->t);
    if (workspace && ((uintptr_t)workspace & 255))
        return fail(h, LBEM_ERR_ARG, "workspace must be 256-byte aligned");
    const AdjLayout L = adj_layout(h, n_steps, K);
    if (workspace && workspace_bytes < L.total)
        return fail(h, LBEM_ERR_OOM, "adjoint workspace of %zu bytes is smaller than the %zu needed",
                    workspace_bytes, L.total);
    h->adj_valid = false;
    if (h->adj_owns && h->adj_ws) {
        CK(h, cudaStreamSynchronize(h->stream));
        cudaFree(h->adj_ws);
    }
    h->adj_ws = nullptr;
    h->adj_owns = false;
    if (workspace) {
        h->adj_ws = (char *)workspace;
        h->adj_bytes = workspace_bytes;
    } else {
        cudaError_t e = cudaMalloc((void **)&h->adj_ws, L.total);
        if (e != cudaSuccess) {
            cudaGetLastError();
            h->adj_ws = nullptr;
            return fail(h, LBEM_ERR_OOM, "cudaMalloc of %zu bytes failed: %s", L.total, cudaGetErrorString(e));
        }
        h->adj_owns = true;
        h->adj_bytes = L.total;
    }
    const size_t pop = (size_t)h->Q * h->P * 4;
    const size_t line = (size_t)h->Q * h->n_line_max * 4;
    for (int seg = 0; seg < L.nseg; ++seg) {
        char *ck = h->adj_ws + L.ck0 + (size_t)seg * L.ck_stride;
        CK(h, cudaMemcpyAsync(ck, h->f[h->cur], pop, cudaMemcpyDeviceToDevice, h->stream));
        // the replay keeps line(t) in buffer t mod 3
        const int64_t t0 = (int64_t)seg * K;
        for (int k = 0; k < 3; ++k)
            CK(h, cudaMemcpyAsync(ck + L.ck_lines + (size_t)((t0 + k) % 3) * align256(line), line_at(h, t0 + k),
                                  line, cudaMemcpyDeviceToDevice, h->stream));
        const int64_t len = std::min<int64_t>(K, n_steps - (int64_t)seg * K);
        const int rc = lbem_step(h, len);
        if (rc != LBEM_OK) return rc;
    }
    h->adj_steps = n_steps;
    h->adj_K = K;
    h->adj_valid = true;
    return LBEM_OK;
}

int32_t lbem_adjoint(lbem_handle h, const double *theta, const double *phi, const double *weights,
                     int32_t n_ang, float *grad_out, int32_t grad_on_device, double *J_out)
{
    if (!h) return fail(nullptr, LBEM_ERR_ARG, "NULL handle");
    if (h->aa) return fail(h, LBEM_ERR_ARG, "the adjoint needs two population buffers (not in-place streaming)");
    if (!h->adj_valid)
        return fail(h, LBEM_ERR_STATE, "no checkpointed forward run for the current permittivity and window");
    if (n_ang < 1 || n_ang > kAngleBatch || !theta || !weights || !grad_out)
        return fail(h, LBEM_ERR_ARG, "need 1..%d angles with theta, weights and grad_out", kAngleBatch);
    if (h->g.mode == 2 && !phi) return fail(h, LBEM_ERR_ARG, "3D needs phi");
    const int64_t w_end = h->dft_t0 + (int64_t)h->dft_periods * h->T - 1;  // last field time in the window
    if (h->dft_t0 < 1 || w_end > h->adj_steps || w_end > h->t)
        return fail(h, LBEM_ERR_STATE, "the DFT window must lie inside the checkpointed run");
    const AdjLayout L = adj_layout(h, h->adj_steps, h->adj_K);
    char *W = h->adj_ws;
    const int NE = h->g.mode == 0 ? 1 : (h->g.mode == 1 ? 2 : 3);
    const size_t pop = (size_t)h->Q * h->P * 4;
    const size_t line = (size_t)h->Q * h->n_line_max * 4;

    // 1. far field of the angles: N, L and |S|^2
    FarFieldArgs fa;
    std::memset(&fa, 0, sizeof fa);
    fa.dft = h->dft;
    fa.line_dft = h->line_dft;
    fa.g = h->faces;
    fa.mode = h->g.mode;
    fa.k = 2.0 * M_PI / h->wave.wavelength;
    for (int c = 0; c < 3; ++c) {
        fa.center[c] = h->wave.center[c];
        fa.pol[c] = h->wave.pol[c];
    }
    centre_nodes(h, &fa.center_i0, &fa.center_i1);
    fa.chunks = far_field_chunks(h->faces);
    double *d_theta = h->scratch;
    double *d_phi = d_theta + kAngleBatch;
    double *d_s2 = d_phi + kAngleBatch;
    double *d_amp = d_s2 + kAngleBatch;
    double *d_part = d_amp + (size_t)kAngleBatch * 12;
    CK(h, cudaMemcpyAsync(d_theta, theta, n_ang * 8, cudaMemcpyHostToDevice, h->stream));
    if (h->g.mode == 2) CK(h, cudaMemcpyAsync(d_phi, phi, n_ang * 8, cudaMemcpyHostToDevice, h->stream));
    double *d_w = (double *)(W + L.wts);
    CK(h, cudaMemcpyAsync(d_w, weights, n_ang * 8, cudaMemcpyHostToDevice, h->stream));
    fa.theta = d_theta;
    fa.phi = d_phi;
    fa.n_ang = n_ang;
    fa.partial = d_part;
    fa.s2 = d_s2;
    fa.amp = d_amp;
    set_far_field_f32(h, fa);
    int l = 0;
    CK(h, launch_far_field(fa, h->stream, &l));
    h->launches += l;

    // 2. dJ/dX of every DFT entry
    AdjWeightArgs wa;
    std::memset(&wa, 0, sizeof wa);
    wa.g = h->faces;
    wa.mode = h->g.mode;
    wa.n_ang = n_ang;
    wa.theta = d_theta;
    wa.phi = d_phi;
    wa.weights = d_w;
    wa.amp = d_amp;
    wa.line_dft = h->line_dft;
    wa.k = fa.k;
    for (int c = 0; c < 3; ++c) {
        wa.center[c] = fa.center[c];
        wa.pol[c] = fa.pol[c];
    }
    wa.center_i0 = fa.center_i0;
    wa.center_i1 = fa.center_i1;
    wa.gamma = (double *)(W + L.gamma);
    wa.G = (double *)(W + L.G);
    CK(h, cudaMemsetAsync(wa.G, 0, h->dft_doubles * 8, h->stream));
    CK(h, launch_adjoint_weights(wa, h->stream, &l));
    h->launches += l;

    // 3. segments backwards: replay the forward run from the checkpoint with
    //    D^F recorded, then the adjoint steps of the segment
    float *mu[2] = {(float *)(W + L.mu[0]), (float *)(W + L.mu[1])};
    float *rf[2] = {(float *)(W + L.rf[0]), (float *)(W + L.rf[1])};
    float *rline[3] = {(float *)(W + L.rline[0]), (float *)(W + L.rline[1]), (float *)(W + L.rline[2])};
    float *rec = (float *)(W + L.rec);
    double *grad = (double *)(W + L.grad);
    CK(h, cudaMemsetAsync(mu[0], 0, pop, h->stream));
    CK(h, cudaMemsetAsync(grad, 0, (size_t)h->P * 8, h->stream));
    int mcur = 0;
    const double scale = 2.0 / ((double)h->dft_periods * h->T);

    StepArgs a;
    fill_common_args(h, a);
    a.dft_on = 0;
    AdjointArgs b;
    std::memset(&b, 0, sizeof b);
    b.inv_eps = h->inv_eps;
    b.grad = grad;
    b.nx = h->g.nx; b.ny = h->g.ny; b.nz = h->g.nz; b.nxp = h->nxp;
    b.P = h->P;
    b.w = h->g.absorber_width;
    b.sigma_max = (float)h->g.sigma_max;
    b.inv_w = b.w > 0 ? 1.0f / (float)b.w : 0.f;
    for (int k = 0; k < 3; ++k) {
        b.nt_lo[k] = h->wave.ntff_lo[k];
        b.nt_hi[k] = h->wave.ntff_hi[k];
    }
    b.G = wa.G;
    for (int f = 0; f < h->faces.nfaces; ++f) {
        b.face_off[f] = h->faces.off[f];
        b.face_nu[f] = h->faces.nu[f];
        b.face_nv[f] = h->faces.nv[f];
    }
    b.dft_scale = scale;

    // phase timing: events before the replay, between replay and backward, after
    std::vector<cudaEvent_t> ev((size_t)3 * L.nseg, nullptr);
    struct EventGuard {
        std::vector<cudaEvent_t> &v;
        ~EventGuard() { for (cudaEvent_t e : v) if (e) cudaEventDestroy(e); }
    } guard{ev};
    for (auto &e : ev) CK(h, cudaEventCreate(&e));
    for (int seg = L.nseg - 1; seg >= 0; --seg) {
        const int64_t t0 = (int64_t)seg * h->adj_K;
        CK(h, cudaEventRecord(ev[3 * seg], h->stream));
        const int64_t len = std::min<int64_t>(h->adj_K, h->adj_steps - t0);
        const char *ck = W + L.ck0 + (size_t)seg * L.ck_stride;
        CK(h, cudaMemcpyAsync(rf[0], ck, pop, cudaMemcpyDeviceToDevice, h->stream));
        for (int k = 0; k < 3; ++k)
            CK(h, cudaMemcpyAsync(rline[k], ck + L.ck_lines + k * align256(line), line,
                                  cudaMemcpyDeviceToDevice, h->stream));
        for (int64_t k = 0; k < len; ++k) {
            const int64_t t = t0 + k;   // state time before the step
            for (int q = 0; q < h->Q; ++q) {
                a.fin_q[q] = rf[k & 1] + (size_t)q * h->P;
                a.fout_q[q] = rf[(k & 1) ^ 1] + (size_t)q * h->P;
            }
            a.line_n = rline[t % 3];
            a.line_n1 = rline[(t + 1) % 3];
            a.line_out = rline[(t + 2) % 3];
            source_fields(h, t + 2, a.src_E, a.src_H);
            a.rec = rec + (size_t)k * NE * h->P;
            cudaError_t e = launch_step_record(h->g.mode, a, h->stream);
            if (e != cudaSuccess) return cuda_fail(h, e, "replay step launch");
            h->launches += 1;
        }
        CK(h, cudaEventRecord(ev[3 * seg + 1], h->stream));
        for (int64_t k = len - 1; k >= 0; --k) {
            const int64_t tf = t0 + k + 1;   // time of the fields of this step
            for (int q = 0; q < h->Q; ++q) {
                b.lin_q[q] = mu[mcur] + (size_t)q * h->P;
                b.lout_q[q] = mu[mcur ^ 1] + (size_t)q * h->P;
            }
            b.rec = rec + (size_t)k * NE * h->P;
            b.dft_on = tf >= h->dft_t0 && tf <= w_end;
            if (b.dft_on) {
                const double ph = 2.0 * M_PI * (double)(tf % h->T) / (double)h->T;
                b.dft_c = std::cos(ph);
                b.dft_s = std::sin(ph);
            }
            cudaError_t e = launch_adjoint_step(h->g.mode, b, h->stream);
            if (e != cudaSuccess) return cuda_fail(h, e, "adjoint step launch");
            h->launches += 1;
            mcur ^= 1;
        }
        CK(h, cudaEventRecord(ev[3 * seg + 2], h->stream));
    }

    // 4. dJ/deps_r and J
    float *out = grad_on_device ? grad_out : h->stage;
    CK(h, launch_adjoint_finalize(grad, h->inv_eps, h->g.nx, h->g.ny, h->g.nz, h->nxp, out, h->stream));
    h->launches += 1;
    if (!grad_on_device)
        CK(h, cudaMemcpyAsync(grad_out, h->stage, (size_t)h->ncell * 4, cudaMemcpyDeviceToHost, h->stream));
    std::vector<double> s2(n_ang);
    CK(h, cudaMemcpyAsync(s2.data(), d_s2, n_ang * 8, cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    h->adj_replay_ms = h->adj_backward_ms = 0.0;
    for (int seg = 0; seg < L.nseg; ++seg) {
        float r = 0.f, b2 = 0.f;
        CK(h, cudaEventElapsedTime(&r, ev[3 * seg], ev[3 * seg + 1]));
        CK(h, cudaEventElapsedTime(&b2, ev[3 * seg + 1], ev[3 * seg + 2]));
        h->adj_replay_ms += r;
        h->adj_backward_ms += b2;
    }
    if (J_out) {
        double J = 0.0;
        for (int i = 0; i < n_ang; ++i) J += weights[i] * s2[i];
        *J_out = J;
    }
    return check_status(h);
}

int32_t lbem_adjoint_timing(lbem_handle h, double *replay_ms, double *backward_ms)
{
    if (!h || !replay_ms || !backward_ms) return fail(h, LBEM_ERR_ARG, "NULL argument");
    *replay_ms = h->adj_replay_ms;
    *backward_ms = h->adj_backward_ms;
    return LBEM_OK;
}

const char *lbem_last_error(lbem_handle h) { return h ? h->err : g_create_err; }

int64_t lbem_kernel_launches(lbem_handle h) { return h ? h->launches : 0; }

}  // extern "C"
