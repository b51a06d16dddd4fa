// lbem_far_field_noalloc: the far-field projection with its scratch in a
// fixed device array, for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc (or any allocator): a host application
// that owns the whole device memory budget and hands plugins fixed buffers, a
// real-time loop where allocation latency is not allowed, or code running
// under a pool whose allocations must not grow.  For them this entry point
// takes every input and output as caller-owned device memory and keeps the
// only scratch it needs -- the per-block partial sums of the projection -- in
// a file-scope __device__ array that every GPU loading the library holds
// until the process exits.
#include <cmath>
#include <cstring>
#include <mutex>

#include "../../include/lbem.h"
#include "lbem_internal.cuh"

namespace lbem {
void set_noctx_error(const char *msg);
}

using namespace lbem;

namespace {

constexpr int kNoAllocChunks = 16;            // face-cell chunks per angle

// Partial sums [angle][chunk][12]: 1024 x 16 x 12 doubles = 1.5 MB per device.
__device__ __align__(256) double g_far_field_scratch[LBEM_NOALLOC_MAX_ANGLES * kNoAllocChunks * 12];

std::mutex g_setup_mutex;
double *g_scratch_dev[kMaxDevices] = {};      // device address of the array, per device

// The array's name is only a host-side stand-in; its device address comes from
// cudaGetSymbolAddress, once per device with that device current.
cudaError_t scratch_of_current_device(double **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_dev[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_far_field_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_dev[dev] = static_cast<double *>(p);
    }
    *out = g_scratch_dev[dev];
    return cudaSuccess;
}

// Eq. 5 (3D) / Eq. 6 (2D) from the chunk partial sums, with |E_I| given.
__global__ void far_field_finalize_given(const FarFieldArgs a, double e_inc)
{
    const int ang = blockIdx.x * blockDim.x + threadIdx.x;
    if (ang >= a.n_ang) return;
    double v[12];
    for (int m = 0; m < 12; ++m) v[m] = 0.0;
    for (int c = 0; c < a.chunks; ++c)
        for (int m = 0; m < 12; ++m) v[m] += a.partial[((long long)ang * a.chunks + c) * 12 + m];
    const double th = a.theta[ang], k = a.k;
    double s2;
    if (a.mode == 2) {
        const double ph = a.phi[ang];
        const double st = sin(th), ct = cos(th), sp = sin(ph), cp = cos(ph);
        const double tv[3] = {ct * cp, ct * sp, -st}, pv[3] = {-sp, cp, 0.0};
        double Nt[2] = {0, 0}, Np[2] = {0, 0}, Lt[2] = {0, 0}, Lp[2] = {0, 0};
        for (int c = 0; c < 3; ++c)
            for (int r = 0; r < 2; ++r) {
                Nt[r] += tv[c] * v[2 * c + r];
                Np[r] += pv[c] * v[2 * c + r];
                Lt[r] += tv[c] * v[6 + 2 * c + r];
                Lp[r] += pv[c] * v[6 + 2 * c + r];
            }
        const double a1r = Nt[0] + Lp[0], a1i = Nt[1] + Lp[1];
        const double a2r = Np[0] - Lt[0], a2i = Np[1] - Lt[1];
        s2 = k * k * k * k * (a1r * a1r + a1i * a1i + a2r * a2r + a2i * a2i) /
             (16.0 * M_PI * M_PI * e_inc * e_inc);
    } else {
        const double pv[3] = {-sin(th), cos(th), 0.0};
        double Np[2] = {0, 0}, Lp[2] = {0, 0};
        for (int c = 0; c < 3; ++c)
            for (int r = 0; r < 2; ++r) {
                Np[r] += pv[c] * v[2 * c + r];
                Lp[r] += pv[c] * v[6 + 2 * c + r];
            }
        double ar, ai;
        if (a.mode == 0) { ar = v[4] - Lp[0]; ai = v[5] - Lp[1]; }   // N_z - L_phi
        else { ar = Np[0] + v[10]; ai = Np[1] + v[11]; }             // N_phi + L_z
        s2 = k * k * (ar * ar + ai * ai) / (8.0 * M_PI * e_inc * e_inc);
    }
    a.s2[ang] = s2;
    if (a.amp)
        for (int m = 0; m < 12; ++m) a.amp[(long long)ang * 12 + m] = v[m];
}

int arg_error(const char *msg)
{
    set_noctx_error(msg);
    return LBEM_ERR_ARG;
}

// Whether p is device (or managed) memory of the current device: a host
// pointer handed to the kernels would fault, or on a system where the GPU can
// read host memory silently be used.  The query allocates nothing.
bool on_current_device(const void *p)
{
    if (!p) return true;
    int dev = 0;
    cudaPointerAttributes at;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();  // clear the sticky-free error of the query
        return false;
    }
    return (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged) && at.device == dev;
}

}  // namespace

extern "C" int32_t lbem_far_field_noalloc(const lbem_ntff_desc *d, const double *dft_dev,
                                          const double *theta_dev, const double *phi_dev,
                                          int32_t n, double *s2_dev, double *amp_dev,
                                          void *cuda_stream)
{
    if (!d) return arg_error("lbem_far_field_noalloc: desc is NULL");
    if (d->mode < 0 || d->mode > 2) return arg_error("lbem_far_field_noalloc: unknown mode");
    const int n3[3] = {d->nx, d->ny, d->nz};
    if (d->nx < 1 || d->ny < 1 || d->nz < 1 || (d->mode != 2 && d->nz != 1) || (d->mode == 2 && d->nz < 2))
        return arg_error("lbem_far_field_noalloc: bad grid extents for the mode");
    for (int ax = 0; ax < 3; ++ax)
        if (d->ntff_lo[ax] < 0 || d->ntff_lo[ax] > d->ntff_hi[ax] || d->ntff_hi[ax] >= n3[ax])
            return arg_error("lbem_far_field_noalloc: NTFF box outside the grid");
    if (!(d->wavelength > 0) || !(d->incident_amplitude > 0) || !std::isfinite(d->incident_amplitude))
        return arg_error("lbem_far_field_noalloc: wavelength and incident_amplitude must be positive");
    if (n < 0 || n > LBEM_NOALLOC_MAX_ANGLES)
        return arg_error("lbem_far_field_noalloc: n must be in [0, LBEM_NOALLOC_MAX_ANGLES = 1024] "
                         "(the fixed scratch holds the partial sums of 1024 angles)");
    if (n == 0) return LBEM_OK;
    if (!dft_dev || !theta_dev || !s2_dev || (d->mode == 2 && !phi_dev))
        return arg_error("lbem_far_field_noalloc: NULL input or output");
    if (!on_current_device(dft_dev) || !on_current_device(theta_dev) || !on_current_device(s2_dev) ||
        (d->mode == 2 && !on_current_device(phi_dev)) || !on_current_device(amp_dev))
        return arg_error("lbem_far_field_noalloc: inputs and outputs must be device memory of the current device");

    double *scratch = nullptr;
    cudaError_t e = scratch_of_current_device(&scratch);
    if (e != cudaSuccess) {
        set_noctx_error(cudaGetErrorString(e));
        return LBEM_ERR_CUDA;
    }

    // face geometry of the documented DFT layout (lbem_get_dft)
    FarFieldArgs a;
    std::memset(&a, 0, sizeof a);
    const int NC = d->mode == 2 ? 6 : 3;
    long long off = 0, cells = 0;
    for (int ax = 0; ax < 3; ++ax) {
        a.g.lo[ax] = d->ntff_lo[ax];
        a.g.hi[ax] = d->ntff_hi[ax];
    }
    for (int ax = 0; ax < 3; ++ax) {
        if (n3[ax] <= 1) continue;
        const int ua = ax == 2 ? 1 : 2, va = ax == 0 ? 1 : 0;
        const int nu = d->ntff_hi[ua] - d->ntff_lo[ua] + 1, nv = d->ntff_hi[va] - d->ntff_lo[va] + 1;
        for (int side = 0; side < 2; ++side) {
            const int f = a.g.nfaces++;
            a.g.axis[f] = ax;
            a.g.side[f] = side;
            a.g.nu[f] = nu;
            a.g.nv[f] = nv;
            a.g.off[f] = off;
            a.g.cell_start[f] = cells;
            off += (long long)NC * 2 * nu * nv;
            cells += (long long)nu * nv;
        }
    }
    a.g.cell_start[a.g.nfaces] = cells;
    a.dft = dft_dev;
    a.mode = d->mode;
    a.n_ang = n;
    a.theta = theta_dev;
    a.phi = phi_dev;
    a.k = 2.0 * M_PI / d->wavelength;
    for (int c = 0; c < 3; ++c) a.center[c] = d->center[c];
    a.chunks = kNoAllocChunks;
    a.partial = scratch;  // every slot is written before it is read: nothing to clear
    a.s2 = s2_dev;
    a.amp = amp_dev;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    e = launch_far_field_partial(a, s);
    if (e == cudaSuccess) {
        far_field_finalize_given<<<(n + 127) / 128, 128, 0, s>>>(a, d->incident_amplitude);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) {
        set_noctx_error(cudaGetErrorString(e));
        return LBEM_ERR_CUDA;
    }
    return LBEM_OK;
}
