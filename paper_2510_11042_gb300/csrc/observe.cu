// Observables and data movement of liblbem:
//   * the FP64 near-to-far-field projection (Sec. 2.4, Eqs. 7-10 in the
//     far-field limit) and the angular intensity |S|^2 (Sec. 2.3, Eqs. 5-6);
//   * the field-energy monitor (Sec. 3.2: steady state is checked by the total
//     field energy) with its non-finite check;
//   * fields of the stored state, permittivity upload, population pack/unpack.
#include <algorithm>
#include <cstring>
#include <mutex>
#include <type_traits>

#include "lbem_internal.cuh"

namespace lbem {
namespace {

template <class S> __device__ __forceinline__ float ldv(const S *p);
template <> __device__ __forceinline__ float ldv<float>(const float *p) { return *p; }
template <> __device__ __forceinline__ float ldv<__half>(const __half *p) { return __half2float(*p); }
template <> __device__ __forceinline__ float ldv<__nv_bfloat16>(const __nv_bfloat16 *p) {
    return __bfloat162float(*p);
}
template <class S> __device__ __forceinline__ void stv(S *p, float v);
template <> __device__ __forceinline__ void stv<float>(float *p, float v) { *p = v; }
template <> __device__ __forceinline__ void stv<__half>(__half *p, float v) { *p = __float2half_rn(v); }
template <> __device__ __forceinline__ void stv<__nv_bfloat16>(__nv_bfloat16 *p, float v) {
    *p = __float2bfloat16_rn(v);
}

__device__ __forceinline__ double warp_sum(double v)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// ------------------------------------------------------------ far field
// Stage 1: one block per (chunk, angle) sums w J e^{j phi}, w M e^{j phi} over
// its share of the face cells; writes 12 doubles (Re/Im of N_xyz, L_xyz).
// acc += w e^{j phi} (J, M) of one face cell with outward normal sgn * e_AX,
// J = n x H, M = -n x E; (e_AX x V)_b1 = -V_b2, (e_AX x V)_b2 = V_b1.
template <int MODE, int AX>
__device__ __forceinline__ void face_cell(const double *base, long long plane, double sgn, double wc,
                                          double ws, double acc[12])
{
    constexpr int b1 = (AX + 1) % 3, b2 = (AX + 2) % 3;
    auto ld = [&](int slot, double &re, double &im) {
        if (slot < 0) { re = 0.0; im = 0.0; }
        else { re = base[(2 * slot) * plane]; im = base[(2 * slot + 1) * plane]; }
    };
    double Hr1, Hi1, Hr2, Hi2, Er1, Ei1, Er2, Ei2;
    ld(slot_H(MODE, b1), Hr1, Hi1);
    ld(slot_H(MODE, b2), Hr2, Hi2);
    ld(slot_E(MODE, b1), Er1, Ei1);
    ld(slot_E(MODE, b2), Er2, Ei2);
    // J_b1 = -sgn H_b2, J_b2 = sgn H_b1, M_b1 = sgn E_b2, M_b2 = -sgn E_b1
    const double J1r = -sgn * Hr2, J1i = -sgn * Hi2, J2r = sgn * Hr1, J2i = sgn * Hi1;
    const double M1r = sgn * Er2, M1i = sgn * Ei2, M2r = -sgn * Er1, M2i = -sgn * Ei1;
    acc[2 * b1 + 0] += J1r * wc - J1i * ws;
    acc[2 * b1 + 1] += J1r * ws + J1i * wc;
    acc[2 * b2 + 0] += J2r * wc - J2i * ws;
    acc[2 * b2 + 1] += J2r * ws + J2i * wc;
    acc[6 + 2 * b1 + 0] += M1r * wc - M1i * ws;
    acc[6 + 2 * b1 + 1] += M1r * ws + M1i * wc;
    acc[6 + 2 * b2 + 0] += M2r * wc - M2i * ws;
    acc[6 + 2 * b2 + 1] += M2r * ws + M2i * wc;
}

constexpr int kFFThreads = 256;
constexpr int kFFTableMax = 4096;   // phase-table entries held in shared memory (64 KB)

// The far-field phase factorises over the coordinates of a face cell,
//   exp(j k r.(p - c)) = prod_a exp(j k r_a (p_a - c_a)),
// so with TABLES each block (one angle) first tabulates exp(j k r_a (p_a - c_a))
// for every coordinate of the NTFF box along the three axes in shared memory,
// and each (cell, angle) pair then costs two complex products instead of an
// FP64 sincos.  Without TABLES (very large boxes) the phase is evaluated
// directly.
template <int MODE, bool TABLES>
__global__ void __launch_bounds__(kFFThreads) far_field_partial(const FarFieldArgs a)
{
    extern __shared__ double tab[];  // [2 * (n0 + n1 + n2)] (re, im)
    const int ang = blockIdx.y;
    const int chunk = blockIdx.x;
    const double th = a.theta[ang];
    double rh[3];
    if (MODE == 2) {
        const double ph = a.phi[ang];
        rh[0] = sin(th) * cos(ph);
        rh[1] = sin(th) * sin(ph);
        rh[2] = cos(th);
    } else {
        rh[0] = cos(th);
        rh[1] = sin(th);
        rh[2] = 0.0;
    }
    int toff[3];
    if (TABLES) {
        const int n0 = a.g.hi[0] - a.g.lo[0] + 1, n1 = a.g.hi[1] - a.g.lo[1] + 1,
                  n2 = a.g.hi[2] - a.g.lo[2] + 1;
        toff[0] = 0;
        toff[1] = n0;
        toff[2] = n0 + n1;
        for (int e = threadIdx.x; e < n0 + n1 + n2; e += blockDim.x) {
            const int ax = e < n0 ? 0 : (e < n0 + n1 ? 1 : 2);
            const double pos = a.g.lo[ax] + (e - toff[ax]);
            double sp, cp;
            sincos(a.k * rh[ax] * (pos - a.center[ax]), &sp, &cp);
            tab[2 * e] = cp;
            tab[2 * e + 1] = sp;
        }
        __syncthreads();
    }
    const long long total = a.g.cell_start[a.g.nfaces];
    const long long per = (total + a.chunks - 1) / a.chunks;
    const long long j0 = (long long)chunk * per;
    const long long j1 = min(total, j0 + per);

    double acc[12];
#pragma unroll
    for (int m = 0; m < 12; ++m) acc[m] = 0.0;

    for (long long j = j0 + threadIdx.x; j < j1; j += blockDim.x) {
        int f = 0;
        while (f + 1 < a.g.nfaces && j >= a.g.cell_start[f + 1]) ++f;
        const long long jl = j - a.g.cell_start[f];
        const int nu = a.g.nu[f], nv = a.g.nv[f];
        const int iu = (int)(jl / nv), iv = (int)(jl % nv);
        const int ax = a.g.axis[f];
        const int ua = ax == 2 ? 1 : 2, va = ax == 0 ? 1 : 0;
        // trapezoidal weights: 1/2 on the edges of each face
        double w = 1.0;
        if (nu > 1 && (iu == 0 || iu == nu - 1)) w *= 0.5;
        if (nv > 1 && (iv == 0 || iv == nv - 1)) w *= 0.5;
        double cp, sp;
        if (TABLES) {
            const int iw = a.g.side[f] ? a.g.hi[ax] - a.g.lo[ax] : 0;
            const double *tw = tab + 2 * (toff[ax] + iw);
            const double *tu = tab + 2 * (toff[ua] + iu);
            const double *tv = tab + 2 * (toff[va] + iv);
            const double pr = tu[0] * tv[0] - tu[1] * tv[1];
            const double pi = tu[0] * tv[1] + tu[1] * tv[0];
            cp = pr * tw[0] - pi * tw[1];
            sp = pr * tw[1] + pi * tw[0];
        } else {
            double pos[3];
            pos[ax] = a.g.side[f] ? a.g.hi[ax] : a.g.lo[ax];
            pos[ua] = a.g.lo[ua] + iu;
            pos[va] = a.g.lo[va] + iv;
            const double phase = a.k * (rh[0] * (pos[0] - a.center[0]) + rh[1] * (pos[1] - a.center[1]) +
                                        rh[2] * (pos[2] - a.center[2]));
            sincos(phase, &sp, &cp);
        }
        const double *base = a.dft + a.g.off[f] + jl;
        const long long plane = (long long)nu * nv;
        const double sgn = a.g.side[f] ? 1.0 : -1.0;
        const double wc = w * cp, ws = w * sp;
        if (ax == 0) face_cell<MODE, 0>(base, plane, sgn, wc, ws, acc);
        else if (ax == 1) face_cell<MODE, 1>(base, plane, sgn, wc, ws, acc);
        else face_cell<MODE, 2>(base, plane, sgn, wc, ws, acc);
    }

    __shared__ double red[kFFThreads / 32][12];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int m = 0; m < 12; ++m) {
        const double v = warp_sum(acc[m]);
        if (lane == 0) red[wid][m] = v;
    }
    __syncthreads();
    if (threadIdx.x < 12) {
        double s = 0.0;
        for (int wi = 0; wi < kFFThreads / 32; ++wi) s += red[wi][threadIdx.x];
        a.partial[((long long)ang * a.chunks + chunk) * 12 + threadIdx.x] = s;
    }
}

// Column form of stage 1 (phase tables in shared memory).  The phase of face
// cell (iu, iv) factorises as t_u(iu) t_v(iv) t_w, and so does the
// trapezoidal weight, so one thread takes one face column (fixed iv; the
// threads of a warp read consecutive iv, coalesced) and sums the tangential
// phasors down the column with t_u(iu) w(iu) alone; the column factor
// t_v(iv) w(iv) t_w multiplies the four column sums once, and J = n x H,
// M = -n x E are formed from them.  Per (cell, angle) this is four complex
// multiply-adds.  Blocks stride over chunks of kFFThreads columns.
template <int MODE>
__global__ void __launch_bounds__(kFFThreads) far_field_columns(const FarFieldArgs a)
{
    extern __shared__ double tab[];  // [2 * (n0 + n1 + n2)] (re, im)
    const int ang = blockIdx.y;
    const double th = a.theta[ang];
    double rh[3];
    if (MODE == 2) {
        const double ph = a.phi[ang];
        rh[0] = sin(th) * cos(ph);
        rh[1] = sin(th) * sin(ph);
        rh[2] = cos(th);
    } else {
        rh[0] = cos(th);
        rh[1] = sin(th);
        rh[2] = 0.0;
    }
    const int n0 = a.g.hi[0] - a.g.lo[0] + 1, n1 = a.g.hi[1] - a.g.lo[1] + 1,
              n2 = a.g.hi[2] - a.g.lo[2] + 1;
    const int toff[3] = {0, n0, n0 + n1};
    for (int e = threadIdx.x; e < n0 + n1 + n2; e += blockDim.x) {
        const int ax = e < n0 ? 0 : (e < n0 + n1 ? 1 : 2);
        const double pos = a.g.lo[ax] + (e - toff[ax]);
        double sp, cp;
        sincos(a.k * rh[ax] * (pos - a.center[ax]), &sp, &cp);
        tab[2 * e] = cp;
        tab[2 * e + 1] = sp;
    }
    __syncthreads();

    int ncols = 0;
    for (int f = 0; f < a.g.nfaces; ++f) ncols += a.g.nv[f];
    double acc[12];
#pragma unroll
    for (int m = 0; m < 12; ++m) acc[m] = 0.0;

    for (int col = blockIdx.x * kFFThreads + threadIdx.x; col < ncols; col += a.chunks * kFFThreads) {
        int f = 0, iv = col;
        while (iv >= a.g.nv[f]) iv -= a.g.nv[f++];
        const int nu = a.g.nu[f], nv = a.g.nv[f];
        const int ax = a.g.axis[f];
        const int ua = ax == 2 ? 1 : 2, va = ax == 0 ? 1 : 0;
        const int b1 = (ax + 1) % 3, b2 = (ax + 2) % 3;
        const int sH1 = slot_H(MODE, b1), sH2 = slot_H(MODE, b2);
        const int sE1 = slot_E(MODE, b1), sE2 = slot_E(MODE, b2);
        const long long plane = (long long)nu * nv;
        const double *base = a.dft + a.g.off[f] + iv;
        const double *tu = tab + 2 * toff[ua];
        // column sums of t_u w_u X for X = H_b1, H_b2, E_b1, E_b2 (re, im)
        double sH1r = 0, sH1i = 0, sH2r = 0, sH2i = 0, sE1r = 0, sE1i = 0, sE2r = 0, sE2i = 0;
        for (int iu = 0; iu < nu; ++iu) {
            double pr = tu[2 * iu], pi = tu[2 * iu + 1];
            if (nu > 1 && (iu == 0 || iu == nu - 1)) {
                pr *= 0.5;
                pi *= 0.5;
            }
            const double *c = base + (long long)iu * nv;
            if (sH1 >= 0) {
                const double xr = c[(2 * sH1) * plane], xi = c[(2 * sH1 + 1) * plane];
                sH1r = fma(pr, xr, fma(-pi, xi, sH1r));
                sH1i = fma(pr, xi, fma(pi, xr, sH1i));
            }
            if (sH2 >= 0) {
                const double xr = c[(2 * sH2) * plane], xi = c[(2 * sH2 + 1) * plane];
                sH2r = fma(pr, xr, fma(-pi, xi, sH2r));
                sH2i = fma(pr, xi, fma(pi, xr, sH2i));
            }
            if (sE1 >= 0) {
                const double xr = c[(2 * sE1) * plane], xi = c[(2 * sE1 + 1) * plane];
                sE1r = fma(pr, xr, fma(-pi, xi, sE1r));
                sE1i = fma(pr, xi, fma(pi, xr, sE1i));
            }
            if (sE2 >= 0) {
                const double xr = c[(2 * sE2) * plane], xi = c[(2 * sE2 + 1) * plane];
                sE2r = fma(pr, xr, fma(-pi, xi, sE2r));
                sE2i = fma(pr, xi, fma(pi, xr, sE2i));
            }
        }
        // column factor t_v(iv) w_v(iv) t_w and the outward normal's sign
        const int iw = a.g.side[f] ? a.g.hi[ax] - a.g.lo[ax] : 0;
        const double *tv = tab + 2 * (toff[va] + iv), *tw = tab + 2 * (toff[ax] + iw);
        double wv = 1.0;
        if (nv > 1 && (iv == 0 || iv == nv - 1)) wv = 0.5;
        const double sgn = a.g.side[f] ? 1.0 : -1.0;
        const double cr = wv * (tv[0] * tw[0] - tv[1] * tw[1]);
        const double ci = wv * (tv[0] * tw[1] + tv[1] * tw[0]);
        // J_b1 = -sgn H_b2, J_b2 = sgn H_b1, M_b1 = sgn E_b2, M_b2 = -sgn E_b1
        auto add = [&](int m, double s, double xr, double xi) {
            acc[m] += s * (cr * xr - ci * xi);
            acc[m + 1] += s * (cr * xi + ci * xr);
        };
        add(2 * b1, -sgn, sH2r, sH2i);
        add(2 * b2, sgn, sH1r, sH1i);
        add(6 + 2 * b1, sgn, sE2r, sE2i);
        add(6 + 2 * b2, -sgn, sE1r, sE1i);
    }

    __shared__ double red[kFFThreads / 32][12];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int m = 0; m < 12; ++m) {
        const double v = warp_sum(acc[m]);
        if (lane == 0) red[wid][m] = v;
    }
    __syncthreads();
    if (threadIdx.x < 12) {
        double s = 0.0;
        for (int wi = 0; wi < kFFThreads / 32; ++wi) s += red[wi][threadIdx.x];
        a.partial[((long long)ang * a.chunks + blockIdx.x) * 12 + threadIdx.x] = s;
    }
}

// Stage 2: one thread per angle; fixed-order sum over chunks, then Eq. 5/6.
__global__ void far_field_finalize(const FarFieldArgs a)
{
    const int ang = blockIdx.x * blockDim.x + threadIdx.x;
    if (ang >= a.n_ang) return;
    double v[12];
    for (int m = 0; m < 12; ++m) v[m] = 0.0;
    for (int c = 0; c < a.chunks; ++c)
        for (int m = 0; m < 12; ++m) v[m] += a.partial[((long long)ang * a.chunks + c) * 12 + m];
    // |E_I|: incident-line E phasor along pol, mean over the two nodes around the centre
    double ei = 0.0;
    const int nodes[2] = {a.center_i0, a.center_i1};
    for (int t = 0; t < 2 && a.ei_fixed <= 0.0; ++t) {
        double re = 0.0, im = 0.0;
        for (int c = 0; c < 3; ++c) {
            re += a.pol[c] * a.line_dft[(nodes[t] * 3 + c) * 2 + 0];
            im += a.pol[c] * a.line_dft[(nodes[t] * 3 + c) * 2 + 1];
        }
        ei += 0.5 * sqrt(re * re + im * im);
    }
    if (a.ei_fixed > 0.0) ei = a.ei_fixed;
    const double th = a.theta[ang];
    const double k = a.k;
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
             (16.0 * M_PI * M_PI * ei * ei);
    } else {
        const double pv[3] = {-sin(th), cos(th), 0.0};
        double Np[2] = {0, 0}, Lp[2] = {0, 0};
        for (int c = 0; c < 3; ++c)
            for (int r = 0; r < 2; ++r) {
                Np[r] += pv[c] * v[2 * c + r];
                Lp[r] += pv[c] * v[6 + 2 * c + r];
            }
        double ar, ai;
        if (a.mode == 0) { ar = v[4] - Lp[0]; ai = v[5] - Lp[1]; }      // N_z - L_phi
        else { ar = Np[0] + v[10]; ai = Np[1] + v[11]; }                // N_phi + L_z
        s2 = k * k * (ar * ar + ai * ai) / (8.0 * M_PI * ei * ei);
    }
    a.s2[ang] = s2;
    if (a.amp)
        for (int m = 0; m < 12; ++m) a.amp[(long long)ang * 12 + m] = v[m];
}

// ------------------------------------------------------------ permittivity
// inv_eps == nullptr: only validate (eps_r finite and >= 1) into *bad.
__global__ void inv_eps_kernel(const float *eps, float *inv_eps, int nx, int ny, int nz, int nxp,
                               int *bad)
{
    const long long n = (long long)nx * ny * nz;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(i % nx);
        const long long r = i / nx;
        const float e = eps[i];
        if (inv_eps == nullptr) {
            if (!(e >= 1.0f) || !isfinite(e)) atomicOr(bad, 1);
        } else {
            inv_eps[r * nxp + x] = 1.0f / e;
        }
    }
}

// ------------------------------------------------------------ pack / unpack
// Incident population of plane q at cell (x, y, z) when it lies in the
// total-field box (where the stored value is the scattered part), else 0.
__device__ __forceinline__ float inc_at(const IncView &v, int q, int x, int y, int z)
{
    if (!v.on) return 0.f;
    if (x < v.tf_lo[0] || x > v.tf_hi[0] || y < v.tf_lo[1] || y > v.tf_hi[1] || z < v.tf_lo[2] ||
        z > v.tf_hi[2])
        return 0.f;
    if (v.on == 2) {
        // vacuum equilibrium (Eq. 2) of the analytic plane wave at the state's time
        const int i = plane_dir(v.mode, q), s = plane_slot(v.mode, q);
        if (i == 0) return 0.f;
        const int ne = mode_NE(v.mode);
        const int c = s < ne ? (v.mode == 0 ? 2 : s) : (v.mode == 1 ? 2 : s - ne);
        const float amp = (float)pw_amplitude(v.pw, x, y, z, v.t);
        const float E[3] = {amp * (float)v.pw.pol[0], amp * (float)v.pw.pol[1], amp * (float)v.pw.pol[2]};
        const float H[3] = {amp * (float)v.pw.kxp[0], amp * (float)v.pw.kxp[1], amp * (float)v.pw.kxp[2]};
        return s < ne ? (E[c] - cross_c(i, H, c)) * (1.0f / 6.0f) : (H[c] + cross_c(i, E, c)) * (1.0f / 6.0f);
    }
    const int s = v.axis == 0 ? x : (v.axis == 1 ? y : z);
    return v.line[(size_t)q * v.n + s];
}

__global__ void fill_kernel(float *p, long long n, float v)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        p[i] = v;
}

// Plane q of the stored populations: element base + w * cell (pop_index).
template <class S>
__global__ void pack_kernel(const S *f, int w, int q, float scale, float *out, int nx, int ny,
                            long long ncell, int nxp, IncView inc)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < ncell;
         i += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(i % nx);
        const long long r = i / nx;
        const int y = (int)(r % ny), z = (int)(r / ny);
        out[i] = ldv<S>(f + w * (r * nxp + x)) * scale + inc_at(inc, q, x, y, z);
    }
}

template <class S>
__global__ void unpack_kernel(S *f, int w, int q, float inv_scale, const float *in, int nx, int ny,
                              long long ncell, int nxp, IncView inc)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < ncell;
         i += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(i % nx);
        const long long r = i / nx;
        const int y = (int)(r % ny), z = (int)(r / ny);
        stv<S>(f + w * (r * nxp + x), (in[i] - inc_at(inc, q, x, y, z)) * inv_scale);
    }
}

// Convert the stored populations of the total-field box between the scattered
// part and the total (sign = +1: add the incident line, -1: remove it).
template <class S>
__global__ void add_incident_kernel(int mode, S *f, long long P, int Q, float scale, int nx, int ny,
                                    long long ncell, int nxp, IncView inc, float sign)
{
    const float inv = 1.0f / scale;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < ncell;
         i += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(i % nx);
        const long long r = i / nx;
        const int y = (int)(r % ny), z = (int)(r / ny);
        for (int q = 0; q < Q; ++q) {
            const float add = inc_at(inc, q, x, y, z);
            if (add == 0.f) continue;
            S *p = f + pop_index(mode, (int)sizeof(S), P, q, r * nxp + x);
            stv<S>(p, (ldv<S>(p) * scale + sign * add) * inv);
        }
    }
}

// Total-field populations of n listed cells (x, y, z triplets): out[k][q].
template <int MODE, class S>
__global__ void probe_kernel(const S *f, float sc, long long P, int ny, int nxp, const int *xyz, int n,
                             IncView inc, float *out)
{
    constexpr int Q = Planes<MODE>::Q;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n * Q; j += gridDim.x * blockDim.x) {
        const int k = j / Q, q = j % Q;
        const int x = xyz[3 * k], y = xyz[3 * k + 1], z = xyz[3 * k + 2];
        const long long c = ((long long)z * ny + y) * nxp + x;
        out[j] = ldv<S>(f + pop_index(MODE, (int)sizeof(S), P, q, c)) * sc + inc_at(inc, q, x, y, z);
    }
}

template <int MODE, class S>
static cudaError_t probe_t(const void *f, float sc, long long P, int ny, int nxp, const int *xyz, int n,
                           const IncView &inc, float *out, cudaStream_t s)
{
    const int total = n * Planes<MODE>::Q;
    probe_kernel<MODE, S><<<(total + 255) / 256, 256, 0, s>>>((const S *)f, sc, P, ny, nxp, xyz, n, inc,
                                                              out);
    return cudaGetLastError();
}

// ------------------------------------------------------------ fields & energy
template <int MODE, class S>
__device__ __forceinline__ void cell_DB(const S *f, float sc, long long P, long long c,
                                        const IncView &inc, int x, int y, int z, float D[3],
                                        float B[3])
{
    using PL = Planes<MODE>;
    D[0] = D[1] = D[2] = 0.f;
    B[0] = B[1] = B[2] = 0.f;
#pragma unroll
    for (int q = 0; q < PL::Q; ++q) {
        const float v = ldv<S>(f + pop_index(MODE, (int)sizeof(S), P, q, c)) * sc + inc_at(inc, q, x, y, z);
        if (PL::fam(q) == 0) D[PL::comp(q)] += v;
        else B[PL::comp(q)] += v;
    }
}

// One field component per launch: comp 0..2 -> E_x..E_z, 3..5 -> H_x..H_z.
template <int MODE, class S>
__global__ void fields_kernel(const S *f, const float *inv_eps, const float *inv_mu, float sc,
                              long long P, int nx, int ny, long long ncell, int nxp, IncView inc,
                              int comp, float *out)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < ncell;
         i += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(i % nx);
        const long long r = i / nx;
        const long long c = r * nxp + x;
        float D[3], B[3];
        cell_DB<MODE, S>(f, sc, P, c, inc, x, (int)(r % ny), (int)(r / ny), D, B);
        out[i] = comp < 3 ? D[comp] * inv_eps[c] : B[comp - 3] * (inv_mu ? inv_mu[c] : 1.0f);
    }
}

constexpr int kEThreads = 256;

template <int MODE, class S>
__global__ void __launch_bounds__(kEThreads) energy_partial(const S *f, const float *inv_eps,
                                                            const float *inv_mu,
                                                            float sc, long long P, int nx, int ny,
                                                            long long ncell, int nxp, IncView inc,
                                                            double *partial)
{
    double acc = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < ncell;
         i += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(i % nx);
        const long long r = i / nx;
        const long long c = r * nxp + x;
        float D[3], B[3];
        cell_DB<MODE, S>(f, sc, P, c, inc, x, (int)(r % ny), (int)(r / ny), D, B);
        const double ie = inv_eps[c], im = inv_mu ? (double)inv_mu[c] : 1.0;
        // 1/2 (eps |E|^2 + mu |H|^2) = 1/2 (|D|^2 / eps + |B|^2 / mu)
        acc += 0.5 * (((double)D[0] * D[0] + (double)D[1] * D[1] + (double)D[2] * D[2]) * ie +
                      ((double)B[0] * B[0] + (double)B[1] * B[1] + (double)B[2] * B[2]) * im);
    }
    __shared__ double red[kEThreads / 32];
    const double v = warp_sum(acc);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < kEThreads / 32; ++w) s += red[w];
        partial[blockIdx.x] = s;
    }
}

__global__ void sum_partials(const double *partial, int n, double *out)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double s = 0.0;
        for (int i = 0; i < n; ++i) s += partial[i];
        *out = s;
    }
}

inline int grid_for(long long n, int threads)
{
    long long b = (n + threads - 1) / threads;
    const long long cap = 32LL * std::max(1, sm_count());
    if (b > cap) b = cap;
    return (int)(b < 1 ? 1 : b);
}


// ---------------------------------------------------------------------------
// 3D far field as an FP32 contraction.  With the phase factorised as above,
// the projection of face f is, per angle a and tangential component X,
//   sum_v t_v(a, v) t_w(a) sum_u t_u(a, u) w_u w_v X(u, v),
// a complex matrix product [angles x u] . [u x (v, X)] followed by a short
// contraction over v.  GB300's FP64 pipe runs at 1/64 of its FP32 rate, so
// the FP64 column kernel above spends ~17 ms on a 384^3 sphere's 543 angles.
// Here the products and the sums over at most uc face rows (and over the 64
// columns of a tile) are FP32, and everything above that (column tiles, row
// chunks, faces) is summed in FP64, in a fixed order.  Phases are evaluated in
// FP64 and rounded once; the phasors are rounded once to FP32.  A term then
// carries ~2^-23 relative error and a partial FP32 sum of n terms at most
// n 2^-24 of its absolute sum (n <= uc = 16..512 rows, or 64 columns).
constexpr int kF32Threads = 256;
constexpr int kF32Angles = 32;   // angles per block: 8 warps x 4
constexpr int kF32Cols = 64;     // face columns per tile: 32 lanes x 2
constexpr int kF32Rows = 16;     // face rows staged in shared memory per pass

// Phase tables tab32[e][a] = exp(j k r_ax(a) (p_e - c_ax)) for the box
// coordinates p_e along x, y, z (e in [0, n0 + n1 + n2)); zero for padded angles.
__global__ void ff32_tables(const FarFieldArgs a)
{
    const int n0 = a.g.hi[0] - a.g.lo[0] + 1, n1 = a.g.hi[1] - a.g.lo[1] + 1,
              n2 = a.g.hi[2] - a.g.lo[2] + 1;
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long long)(n0 + n1 + n2) * a.n_ang_pad) return;
    const int ang = (int)(i % a.n_ang_pad), e = (int)(i / a.n_ang_pad);
    float2 out = make_float2(0.f, 0.f);
    if (ang < a.n_ang) {
        const int ax = e < n0 ? 0 : (e < n0 + n1 ? 1 : 2);
        const int toff = ax == 0 ? 0 : (ax == 1 ? n0 : n0 + n1);
        const double th = a.theta[ang], ph = a.phi[ang];
        const double r = ax == 0 ? sin(th) * cos(ph) : (ax == 1 ? sin(th) * sin(ph) : cos(th));
        const double pos = a.g.lo[ax] + (e - toff);
        double sp, cp;
        sincos(a.k * r * (pos - a.center[ax]), &sp, &cp);
        out = make_float2((float)cp, (float)sp);
    }
    a.tab32[i] = out;
}

// Packed faces x32[f][u][q][v] = w_u w_v X_q(u, v) in FP32, q = H_b1, H_b2,
// E_b1, E_b2 (b1 = AX+1, b2 = AX+2 mod 3); zero in the padding.
__global__ void ff32_pack(const FarFieldArgs a)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.off32[a.g.nfaces]) return;
    int f = 0;
    while (i >= a.off32[f + 1]) ++f;
    const long long r = i - a.off32[f];
    const int nvp = a.nvp[f];
    const int v = (int)(r % nvp);
    const long long t = r / nvp;
    const int q = (int)(t % 4), u = (int)(t / 4);
    const int nu = a.g.nu[f], nv = a.g.nv[f];
    float2 out = make_float2(0.f, 0.f);
    if (u < nu && v < nv) {
        const int ax = a.g.axis[f], b1 = (ax + 1) % 3, b2 = (ax + 2) % 3;
        const int slot = q == 0 ? slot_H(2, b1) : q == 1 ? slot_H(2, b2) : q == 2 ? slot_E(2, b1) : slot_E(2, b2);
        const long long plane = (long long)nu * nv;
        const double *c = a.dft + a.g.off[f] + (long long)u * nv + v;
        double w = 1.0;
        if (nu > 1 && (u == 0 || u == nu - 1)) w *= 0.5;
        if (nv > 1 && (v == 0 || v == nv - 1)) w *= 0.5;
        out = make_float2((float)(w * c[(2 * slot) * plane]), (float)(w * c[(2 * slot + 1) * plane]));
    }
    a.x32[i] = out;
}

__device__ __forceinline__ void cmac(float &sr, float &si, float2 p, float xr, float xi)
{
    sr = fmaf(p.x, xr, fmaf(-p.y, xi, sr));
    si = fmaf(p.x, xi, fmaf(p.y, xr, si));
}

// One step of a reduce-scatter over the warp: a lane keeps the half of its
// values selected by its bit H and adds the partner's copy of that half.
// After the steps 16, 8, 4, 2, 1, lane l holds the warp's sum of value l.
template <int H>
__device__ __forceinline__ void rs_stage(float (&o)[32], int lane)
{
    const bool up = (lane & H) != 0;
#pragma unroll
    for (int i = 0; i < H; ++i) {
        const float send = up ? o[i] : o[i + H];
        const float keep = up ? o[i + H] : o[i];
        o[i] = keep + __shfl_xor_sync(0xffffffffu, send, H);
    }
}

// One block per (tile of 32 angles, chunk of uc rows of one face).  Warp w
// owns angles 4w..4w+3 of the tile and lane l columns 2l, 2l+1 of each
// 64-column tile.  Per column tile: FP32 column sums over the chunk's rows,
// then the column factor, a reduce-scatter over the warp (lane l ends with
// value l of the warp's 4 angles x 8 outputs), and an FP64 add into shared
// memory.  Writes partial[angle][chunk][12].
__global__ void __launch_bounds__(kF32Threads, 2) far_field_f32(const FarFieldArgs a)
{
    extern __shared__ float4 ff_sm[];
    float2 *At = reinterpret_cast<float2 *>(ff_sm);                  // [uc][32] row phases
    float4 *Xs = ff_sm + a.uc * (kF32Angles / 2);                    // [16 rows x 4 q][32] (2 columns)
    double *acc = reinterpret_cast<double *>(Xs + kF32Rows * 4 * 32);  // [32 angles][12]
    const int lane = threadIdx.x & 31, wg = threadIdx.x >> 5;
    const int ang0 = blockIdx.x * kF32Angles;
    const int ch = blockIdx.y;
    int f = 0;
    while (f + 1 < a.g.nfaces && ch >= a.chunk_start[f + 1]) ++f;
    const int u0 = (ch - a.chunk_start[f]) * a.uc;
    const int nu = a.g.nu[f], nv = a.g.nv[f], nvp = a.nvp[f];
    const int un = min(a.uc, a.nup[f] - u0);  // a multiple of kF32Rows
    const int ax = a.g.axis[f];
    const int ua = ax == 2 ? 1 : 2, va = ax == 0 ? 1 : 0;
    const int b1 = (ax + 1) % 3, b2 = (ax + 2) % 3;
    const int n0 = a.g.hi[0] - a.g.lo[0] + 1, n1 = a.g.hi[1] - a.g.lo[1] + 1;
    auto toff = [&](int axis) { return axis == 0 ? 0 : (axis == 1 ? n0 : n0 + n1); };
    const int eu = toff(ua), ev = toff(va);
    for (int i = threadIdx.x; i < un * kF32Angles; i += kF32Threads) {
        const int u = i / kF32Angles, j = i % kF32Angles;
        At[i] = u0 + u < nu ? a.tab32[(long long)(eu + u0 + u) * a.n_ang_pad + ang0 + j]
                            : make_float2(0.f, 0.f);
    }
    for (int i = threadIdx.x; i < kF32Angles * 12; i += kF32Threads) acc[i] = 0.0;
    const int ew = toff(ax) + (a.g.side[f] ? a.g.hi[ax] - a.g.lo[ax] : 0);
    const double sgn = a.g.side[f] ? 1.0 : -1.0;
    const float4 *X = reinterpret_cast<const float4 *>(a.x32 + a.off32[f]);
    const int nvq = nvp / 2;  // float4 (two columns) per row of one component
    // output slot of reduce-scatter value q of an angle: J_b1, J_b2, M_b1, M_b2 (re, im)
    const int qv = lane & 7, jv = lane >> 3;
    const int mslot = (qv < 4 ? 0 : 6) + 2 * ((qv & 2) ? b2 : b1) + (qv & 1);

    for (int c0 = 0; c0 < nvp; c0 += kF32Cols) {
        float sr[4][2][4], si[4][2][4];  // [angle][column][q]
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int c = 0; c < 2; ++c)
#pragma unroll
                for (int q = 0; q < 4; ++q) sr[j][c][q] = si[j][c][q] = 0.f;
        for (int s0 = 0; s0 < un; s0 += kF32Rows) {
            __syncthreads();
            for (int i = threadIdx.x; i < kF32Rows * 4 * 32; i += kF32Threads) {
                const int row = i >> 5, l = i & 31;  // row = us * 4 + q
                Xs[i] = X[(long long)((u0 + s0) * 4 + row) * nvq + c0 / 2 + l];
            }
            __syncthreads();
#pragma unroll 2
            for (int us = 0; us < kF32Rows; ++us) {
                const float4 *pw = reinterpret_cast<const float4 *>(At + (s0 + us) * kF32Angles + 4 * wg);
                const float4 pa = pw[0], pb = pw[1];
                const float2 p[4] = {make_float2(pa.x, pa.y), make_float2(pa.z, pa.w),
                                     make_float2(pb.x, pb.y), make_float2(pb.z, pb.w)};
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const float4 x = Xs[(us * 4 + q) * 32 + lane];
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        cmac(sr[j][0][q], si[j][0][q], p[j], x.x, x.y);
                        cmac(sr[j][1][q], si[j][1][q], p[j], x.z, x.w);
                    }
                }
            }
        }
        // column factor t_v t_w; J_b1 = -H_b2, J_b2 = H_b1, M_b1 = E_b2, M_b2 = -E_b1
        // (times the normal's sign, applied in FP64 below)
        float o[32];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const long long ang = ang0 + 4 * wg + j;
            const float2 tw = a.tab32[(long long)ew * a.n_ang_pad + ang];
#pragma unroll
            for (int q = 0; q < 8; ++q) o[8 * j + q] = 0.f;
#pragma unroll
            for (int c = 0; c < 2; ++c) {
                const int v = c0 + 2 * lane + c;
                const float2 tv = v < nv ? a.tab32[(long long)(ev + v) * a.n_ang_pad + ang]
                                         : make_float2(0.f, 0.f);
                const float cr = tv.x * tw.x - tv.y * tw.y, ci = tv.x * tw.y + tv.y * tw.x;
                const float sg[4] = {1.f, -1.f, -1.f, 1.f};   // sign of q in its output
                const int oq[4] = {2, 0, 6, 4};               // H_b1 -> J_b2, H_b2 -> J_b1, E_b1 -> M_b2, E_b2 -> M_b1
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const float xr = sg[q] * sr[j][c][q], xi = sg[q] * si[j][c][q];
                    o[8 * j + oq[q]] = fmaf(cr, xr, fmaf(-ci, xi, o[8 * j + oq[q]]));
                    o[8 * j + oq[q] + 1] = fmaf(cr, xi, fmaf(ci, xr, o[8 * j + oq[q] + 1]));
                }
            }
        }
        rs_stage<16>(o, lane);
        rs_stage<8>(o, lane);
        rs_stage<4>(o, lane);
        rs_stage<2>(o, lane);
        rs_stage<1>(o, lane);
        acc[(4 * wg + jv) * 12 + mslot] += sgn * (double)o[0];
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kF32Angles * 12; i += kF32Threads) {
        const int j = i / 12, m = i % 12;
        if (ang0 + j < a.n_ang) a.partial[((long long)(ang0 + j) * a.chunks + ch) * 12 + m] = acc[i];
    }
}

}  // namespace

#define LBEM_FF_TABLES(MODE)                                                                 \
    do {                                                                                     \
        if (smem > 48 * 1024) {                                                              \
            cudaError_t e_ = cudaFuncSetAttribute(far_field_columns<MODE>,                   \
                                                  cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                                  kFFTableMax * 2 * (int)sizeof(double));    \
            if (e_ != cudaSuccess) return e_;                                                \
        }                                                                                    \
        far_field_columns<MODE><<<g1, kFFThreads, smem, s>>>(a);                             \
    } while (0)

static size_t ff32_smem(int uc)
{
    return (size_t)uc * kF32Angles * sizeof(float2) + (size_t)kF32Rows * 4 * 32 * sizeof(float4) +
           (size_t)kF32Angles * 12 * sizeof(double);
}

// The 3D projection through far_field_f32: phase tables, packed faces, the
// contraction and the FP64 finalisation.  The chunk height uc (a multiple of
// 16 rows) minimises waves x (uc + 8): fewer, taller chunks waste less per
// block but quantise the grid into more partial waves.
static cudaError_t launch_far_field_f32(FarFieldArgs a, cudaStream_t s, int *launches)
{
    if (a.n_ang <= 0) return cudaSuccess;
    long long off = 0;
    for (int f = 0; f < a.g.nfaces; ++f) {
        a.nup[f] = (a.g.nu[f] + kF32Rows - 1) / kF32Rows * kF32Rows;
        a.nvp[f] = (a.g.nv[f] + kF32Cols - 1) / kF32Cols * kF32Cols;
        a.off32[f] = off;
        off += (long long)a.nup[f] * 4 * a.nvp[f];
    }
    a.off32[a.g.nfaces] = off;
    a.n_ang_pad = (a.n_ang + kF32Angles - 1) / kF32Angles * kF32Angles;
    const int ne = (a.g.hi[0] - a.g.lo[0] + 1) + (a.g.hi[1] - a.g.lo[1] + 1) + (a.g.hi[2] - a.g.lo[2] + 1);
    if (off > a.x32_cap || (long long)ne * a.n_ang_pad > a.tab32_cap) return cudaErrorInvalidValue;
    // resident blocks per SM for each chunk height (shared memory grows with
    // uc), and the shared-memory opt-in: once per device
    constexpr int kMaxUc = 512;
    static std::mutex setup_mu;
    static bool ready_of[kMaxDevices];
    static int per_uc_of[kMaxDevices][kMaxUc / kF32Rows + 1];
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    const int sms = sm_count();
    if (sms < 1) return cudaErrorInvalidDevice;
    int per_uc[kMaxUc / kF32Rows + 1];
    {
        std::lock_guard<std::mutex> lock(setup_mu);
        if (!ready_of[dev]) {
            e = cudaFuncSetAttribute(far_field_f32, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)ff32_smem(kMaxUc));
            for (int uc = kF32Rows; e == cudaSuccess && uc <= kMaxUc; uc += kF32Rows)
                e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_uc_of[dev][uc / kF32Rows], far_field_f32,
                                                                   kF32Threads, ff32_smem(uc));
            if (e != cudaSuccess) return e;
            ready_of[dev] = true;
        }
        std::memcpy(per_uc, per_uc_of[dev], sizeof per_uc);
    }
    const int tiles = a.n_ang_pad / kF32Angles;
    int best_uc = 0;
    double best = 0.0;
    for (int uc = kF32Rows; uc <= kMaxUc; uc += kF32Rows) {
        int chunks = 0;
        for (int f = 0; f < a.g.nfaces; ++f) chunks += (a.nup[f] + uc - 1) / uc;
        const int per = per_uc[uc / kF32Rows];
        if (chunks > kMaxChunks || per < 1) continue;
        const long long blocks = (long long)tiles * chunks;
        const long long waves = (blocks + (long long)per * sms - 1) / ((long long)per * sms);
        const double t = (double)waves * (uc + 8);
        if (best_uc == 0 || t < best) {
            best = t;
            best_uc = uc;
        }
    }
    if (best_uc == 0) return cudaErrorInvalidValue;
    a.uc = best_uc;
    a.chunk_start[0] = 0;
    for (int f = 0; f < a.g.nfaces; ++f) a.chunk_start[f + 1] = a.chunk_start[f] + (a.nup[f] + a.uc - 1) / a.uc;
    a.chunks = a.chunk_start[a.g.nfaces];
    const size_t sm = ff32_smem(a.uc);
    const long long nt = (long long)ne * a.n_ang_pad;
    ff32_tables<<<(unsigned)((nt + 255) / 256), 256, 0, s>>>(a);
    ff32_pack<<<(unsigned)((off + 255) / 256), 256, 0, s>>>(a);
    far_field_f32<<<dim3(tiles, a.chunks), kF32Threads, sm, s>>>(a);
    far_field_finalize<<<(a.n_ang + 127) / 128, 128, 0, s>>>(a);
    if (launches) *launches += 4;
    return cudaGetLastError();
}

cudaError_t launch_far_field(const FarFieldArgs &a, cudaStream_t s, int *launches)
{
    if (a.mode == 2 && a.x32 != nullptr) return launch_far_field_f32(a, s, launches);
    dim3 g1(a.chunks, a.n_ang);
    const int entries = (a.g.hi[0] - a.g.lo[0] + 1) + (a.g.hi[1] - a.g.lo[1] + 1) + (a.g.hi[2] - a.g.lo[2] + 1);
    const bool tables = entries <= kFFTableMax;
    const size_t smem = tables ? (size_t)entries * 2 * sizeof(double) : 0;
    switch (a.mode * 2 + (tables ? 1 : 0)) {
    case 0: far_field_partial<0, false><<<g1, kFFThreads, 0, s>>>(a); break;
    case 1: LBEM_FF_TABLES(0); break;
    case 2: far_field_partial<1, false><<<g1, kFFThreads, 0, s>>>(a); break;
    case 3: LBEM_FF_TABLES(1); break;
    case 4: far_field_partial<2, false><<<g1, kFFThreads, 0, s>>>(a); break;
    case 5: LBEM_FF_TABLES(2); break;
    default: return cudaErrorInvalidValue;
    }
    far_field_finalize<<<(a.n_ang + 127) / 128, 128, 0, s>>>(a);
    if (launches) *launches += 2;
    return cudaGetLastError();
}

// The projection's partial-sum stage alone (the caller finalises).
cudaError_t launch_far_field_partial(const FarFieldArgs &a, cudaStream_t s)
{
    dim3 g1(a.chunks, a.n_ang);
    const int entries = (a.g.hi[0] - a.g.lo[0] + 1) + (a.g.hi[1] - a.g.lo[1] + 1) + (a.g.hi[2] - a.g.lo[2] + 1);
    const bool tables = entries <= kFFTableMax;
    const size_t smem = tables ? (size_t)entries * 2 * sizeof(double) : 0;
    switch (a.mode * 2 + (tables ? 1 : 0)) {
    case 0: far_field_partial<0, false><<<g1, kFFThreads, 0, s>>>(a); break;
    case 1: LBEM_FF_TABLES(0); break;
    case 2: far_field_partial<1, false><<<g1, kFFThreads, 0, s>>>(a); break;
    case 3: LBEM_FF_TABLES(1); break;
    case 4: far_field_partial<2, false><<<g1, kFFThreads, 0, s>>>(a); break;
    case 5: LBEM_FF_TABLES(2); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_fill(float *p, long long n, float v, cudaStream_t s)
{
    fill_kernel<<<grid_for(n, 256), 256, 0, s>>>(p, n, v);
    return cudaGetLastError();
}

cudaError_t launch_inv_eps(const float *eps, float *inv_eps, int nx, int ny, int nz, int nxp,
                           int *bad_flag, cudaStream_t s)
{
    const long long n = (long long)nx * ny * nz;
    inv_eps_kernel<<<grid_for(n, 256), 256, 0, s>>>(eps, inv_eps, nx, ny, nz, nxp, bad_flag);
    return cudaGetLastError();
}

cudaError_t launch_pack(int mode, int storage, const void *f, long long P, int q, float scale,
                        float *out, int nx, int ny, int nz, int nxp, const IncView &inc, cudaStream_t s)
{
    const long long n = (long long)nx * ny * nz;
    const int g = grid_for(n, 256);
    const int eb = storage == 0 ? 4 : 2;
    const long long base = pop_index(mode, eb, P, q, 0);
    const int w = (int)(pop_index(mode, eb, P, q, 1) - base);
    if (storage == 0)
        pack_kernel<float><<<g, 256, 0, s>>>((const float *)f + base, w, q, scale, out, nx, ny, n, nxp, inc);
    else if (storage == 1)
        pack_kernel<__half><<<g, 256, 0, s>>>((const __half *)f + base, w, q, scale, out, nx, ny, n, nxp, inc);
    else
        pack_kernel<__nv_bfloat16><<<g, 256, 0, s>>>((const __nv_bfloat16 *)f + base, w, q, scale, out, nx,
                                                     ny, n, nxp, inc);
    return cudaGetLastError();
}

cudaError_t launch_unpack(int mode, int storage, void *f, long long P, int q, float inv_scale,
                          const float *in, int nx, int ny, int nz, int nxp, const IncView &inc,
                          cudaStream_t s)
{
    const long long n = (long long)nx * ny * nz;
    const int g = grid_for(n, 256);
    const int eb = storage == 0 ? 4 : 2;
    const long long base = pop_index(mode, eb, P, q, 0);
    const int w = (int)(pop_index(mode, eb, P, q, 1) - base);
    if (storage == 0)
        unpack_kernel<float><<<g, 256, 0, s>>>((float *)f + base, w, q, inv_scale, in, nx, ny, n, nxp, inc);
    else if (storage == 1)
        unpack_kernel<__half><<<g, 256, 0, s>>>((__half *)f + base, w, q, inv_scale, in, nx, ny, n, nxp, inc);
    else
        unpack_kernel<__nv_bfloat16><<<g, 256, 0, s>>>((__nv_bfloat16 *)f + base, w, q, inv_scale, in, nx,
                                                       ny, n, nxp, inc);
    return cudaGetLastError();
}

cudaError_t launch_add_incident(int mode, int storage, void *f, long long P, int Q, float scale,
                                int nx, int ny, int nz, int nxp, const IncView &inc, float sign,
                                cudaStream_t s)
{
    const long long n = (long long)nx * ny * nz;
    const int g = grid_for(n, 256);
    if (storage == 0)
        add_incident_kernel<float><<<g, 256, 0, s>>>(mode, (float *)f, P, Q, scale, nx, ny, n, nxp, inc, sign);
    else if (storage == 1)
        add_incident_kernel<__half><<<g, 256, 0, s>>>(mode, (__half *)f, P, Q, scale, nx, ny, n, nxp, inc, sign);
    else
        add_incident_kernel<__nv_bfloat16><<<g, 256, 0, s>>>(mode, (__nv_bfloat16 *)f, P, Q, scale, nx, ny, n,
                                                             nxp, inc, sign);
    return cudaGetLastError();
}

template <int MODE, class S>
static cudaError_t fields_t(const void *f, const float *inv_eps, const float *inv_mu, float sc,
                            long long P, int nx, int ny, int nz, int nxp, const IncView &inc,
                            int comp, float *out, cudaStream_t s)
{
    const long long n = (long long)nx * ny * nz;
    fields_kernel<MODE, S><<<grid_for(n, 256), 256, 0, s>>>((const S *)f, inv_eps, inv_mu, sc, P, nx,
                                                             ny, n, nxp, inc, comp, out);
    return cudaGetLastError();
}

template <int MODE, class S>
static cudaError_t energy_t(const void *f, const float *inv_eps, const float *inv_mu, float sc, long long P,
                            int nx, int ny, int nz, int nxp, const IncView &inc, double *partial,
                            int max_partial, double *out, cudaStream_t s)
{
    const long long n = (long long)nx * ny * nz;
    int g = grid_for(n, kEThreads);
    if (g > max_partial) g = max_partial;
    energy_partial<MODE, S><<<g, kEThreads, 0, s>>>((const S *)f, inv_eps, inv_mu, sc, P, nx, ny, n, nxp,
                                                     inc, partial);
    sum_partials<<<1, 32, 0, s>>>(partial, g, out);
    return cudaGetLastError();
}

#define LBEM_DISPATCH(FN, ...)                                                   \
    switch (mode * 3 + storage) {                                                \
    case 0: return FN<0, float>(__VA_ARGS__);                                    \
    case 1: return FN<0, __half>(__VA_ARGS__);                                   \
    case 2: return FN<0, __nv_bfloat16>(__VA_ARGS__);                            \
    case 3: return FN<1, float>(__VA_ARGS__);                                    \
    case 4: return FN<1, __half>(__VA_ARGS__);                                   \
    case 5: return FN<1, __nv_bfloat16>(__VA_ARGS__);                            \
    case 6: return FN<2, float>(__VA_ARGS__);                                    \
    case 7: return FN<2, __half>(__VA_ARGS__);                                   \
    case 8: return FN<2, __nv_bfloat16>(__VA_ARGS__);                            \
    default: return cudaErrorInvalidValue;                                       \
    }

cudaError_t launch_fields(int mode, int storage, const void *f, const float *inv_eps, const float *inv_mu,
                          float scale, long long P, int nx, int ny, int nz, int nxp,
                          const IncView &inc, int comp, float *out, cudaStream_t s)
{
    LBEM_DISPATCH(fields_t, f, inv_eps, inv_mu, scale, P, nx, ny, nz, nxp, inc, comp, out, s)
}

cudaError_t launch_probe(int mode, int storage, const void *f, float scale, long long P, int ny, int nxp,
                         const int *xyz, int n, const IncView &inc, float *out, cudaStream_t s)
{
    LBEM_DISPATCH(probe_t, f, scale, P, ny, nxp, xyz, n, inc, out, s)
}

cudaError_t launch_energy(int mode, int storage, const void *f, const float *inv_eps, const float *inv_mu,
                          float scale, long long P, int nx, int ny, int nz, int nxp,
                          const IncView &inc, double *partial, int max_partial, double *out,
                          cudaStream_t s, int *launches)
{
    if (launches) *launches += 2;
    LBEM_DISPATCH(energy_t, f, inv_eps, inv_mu, scale, P, nx, ny, nz, nxp, inc, partial, max_partial, out, s)
}

}  // namespace lbem
