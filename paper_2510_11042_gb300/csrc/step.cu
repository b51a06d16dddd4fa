// Fused D3Q7 stream-and-collide step for the lattice-Boltzmann Maxwell scheme
// of arXiv 2510.11042, Sec. 2.1 (Eqs. 1-2) with the outer boundary of Eq. 4.
//
// One launch advances every cell by one time step and, in one extra block,
// the 1D incident line that feeds the total-field/scattered-field links:
//   pull    f_i(r) = f*_i(clamp(r - c_i))           (Eq. 1 streaming + Eq. 4)
//   TF/SF   +/- incident f*_i of the link's source cell on links crossing the box
//   moments D = sum_i e_i, B = sum_i h_i, E = D / eps_r, H = B  (mu_r = 1)
//   DFT     X += x(t) exp(-j w t) on the NTFF box surface (FP64 accumulators)
//   collide f* = 2 f_eq - f (tau = 1/2, equilibria of Eq. 2):
//             e_0* = 2 (eps_r - 1) E - e_0 = 2 (D - E) - e_0
//             e_i* = (E - c_i x H) / 3 - e_i,    h_0* = -h_0,
//             h_i* = (H + c_i x E) / 3 - h_i
//   layer   f* *= 1 - sigma_max (m / W)^3 near the outer faces
//   store   to the other ping-pong buffer.
//
// Memory layout: structure of arrays, one plane per (family, direction,
// component) of nz*ny*nxp elements, x fastest and padded to a multiple of
// 32 elements; 4 B of 1/eps_r per cell.  Each population is read once and
// written once per step: B_cell = 2 Q s + 4 bytes.  The update is a
// memory-bound stencil (~1 flop/byte), so it runs on the CUDA cores; no
// tensor-core path applies.
#include <type_traits>

#include "lbem_internal.cuh"

namespace lbem {
namespace {

template <class S> __device__ __forceinline__ float ld(const S *p);
template <> __device__ __forceinline__ float ld<float>(const float *p) { return __ldg(p); }
template <> __device__ __forceinline__ float ld<__half>(const __half *p) { return __half2float(__ldg(p)); }
template <> __device__ __forceinline__ float ld<__nv_bfloat16>(const __nv_bfloat16 *p) {
    return __bfloat162float(__ldg(p));
}
template <class S> __device__ __forceinline__ void st(S *p, float v);
template <> __device__ __forceinline__ void st<float>(float *p, float v) { *p = v; }
template <> __device__ __forceinline__ void st<__half>(__half *p, float v) { *p = __float2half_rn(v); }
template <> __device__ __forceinline__ void st<__nv_bfloat16>(__nv_bfloat16 *p, float v) {
    *p = __float2bfloat16_rn(v);
}

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

// Moments, collision and equilibrium for one cell held in registers.
template <int MODE>
__device__ __forceinline__ void moments(const float *f, float inv_eps, float D[3], float E[3],
                                        float H[3])
{
    using PL = Planes<MODE>;
    float B[3] = {0.f, 0.f, 0.f};
    D[0] = D[1] = D[2] = 0.f;
#pragma unroll
    for (int q = 0; q < PL::Q; ++q) {
        if (PL::fam(q) == 0) D[PL::comp(q)] += f[q];
        else B[PL::comp(q)] += f[q];
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        E[a] = D[a] * inv_eps;
        H[a] = B[a];
    }
}

template <int MODE>
__device__ __forceinline__ void collide(float *f, const float D[3], const float E[3],
                                        const float H[3])
{
    using PL = Planes<MODE>;
    constexpr float third = 1.0f / 3.0f;
#pragma unroll
    for (int q = 0; q < PL::Q; ++q) {
        const int i = PL::dir(q), a = PL::comp(q);
        float eq2;  // 2 f_eq
        if (PL::fam(q) == 0)
            eq2 = (i == 0) ? 2.f * (D[a] - E[a]) : (E[a] - cross_c(i, H, a)) * third;
        else
            eq2 = (i == 0) ? 0.f : (H[a] + cross_c(i, E, a)) * third;
        f[q] = eq2 - f[q];
    }
}

// Vacuum equilibrium of prescribed fields (hard source of the incident line).
template <int MODE>
__device__ __forceinline__ void vacuum_equilibrium(float *f, const float E[3], const float H[3])
{
    using PL = Planes<MODE>;
    constexpr float sixth = 1.0f / 6.0f;
#pragma unroll
    for (int q = 0; q < PL::Q; ++q) {
        const int i = PL::dir(q), a = PL::comp(q);
        if (i == 0) f[q] = 0.f;
        else if (PL::fam(q) == 0) f[q] = (E[a] - cross_c(i, H, a)) * sixth;
        else f[q] = (H[a] + cross_c(i, E, a)) * sixth;
    }
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

// The 1D incident line: the same update on an n_line x 1 x 1 lattice along
// inc_axis (eps_r = 1), absorbing layer at both ends, hard source at src_index.
template <int MODE>
__device__ void line_update(const StepArgs &a)
{
    using PL = Planes<MODE>;
    constexpr int Q = PL::Q;
    const int n = a.n_line, ax = a.inc_axis;
    for (int s = threadIdx.x; s < n; s += blockDim.x) {
        float f[Q];
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            const int i = PL::dir(q);
            const int c = (dir_axis(i) == ax) ? dir_sign(i) : 0;
            int src = s - c;
            src = src < 0 ? 0 : (src > n - 1 ? n - 1 : src);
            f[q] = a.line_in[(size_t)q * n + src];
        }
        float D[3], E[3], H[3];
        moments<MODE>(f, 1.f, D, E, H);
        if (a.dft_on) {
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const double v = a.dft_scale * (double)E[c];
                a.line_dft[(s * 3 + c) * 2 + 0] += v * a.dft_c;
                a.line_dft[(s * 3 + c) * 2 + 1] -= v * a.dft_s;
            }
        }
        collide<MODE>(f, D, E, H);
        const int d = min(s, n - 1 - s);
        const float keep = layer_keep(d, a.w, a.sigma_max, a.inv_w);
#pragma unroll
        for (int q = 0; q < Q; ++q) f[q] *= keep;
        if (s == a.src_index) vacuum_equilibrium<MODE>(f, a.src_E, a.src_H);
#pragma unroll
        for (int q = 0; q < Q; ++q) a.line_out[(size_t)q * n + s] = f[q];
    }
}

template <int MODE, class S, int BX>
__global__ void __launch_bounds__(BX) step_kernel(const StepArgs a)
{
    using PL = Planes<MODE>;
    constexpr int Q = PL::Q;
    constexpr bool kScaled = !std::is_same<S, float>::value;
    const int b = blockIdx.x;
    if (b >= a.nblk_main) {
        if (a.line_on) line_update<MODE>(a);
        return;
    }
    const int bx = b % a.nblk_x;
    const int row = b / a.nblk_x;
    const int y = row % a.ny;
    const int z = row / a.ny;
    const int x = bx * BX + threadIdx.x;
    if (x >= a.nx) return;

    const int pz = a.ny * a.nxp;
    const int c = z * pz + y * a.nxp + x;
    int src[7];
    src[0] = c;
    src[1] = c - (x > 0 ? 1 : 0);
    src[2] = c + (x < a.nx - 1 ? 1 : 0);
    src[3] = c - (y > 0 ? a.nxp : 0);
    src[4] = c + (y < a.ny - 1 ? a.nxp : 0);
    src[5] = c - (z > 0 ? pz : 0);
    src[6] = c + (z < a.nz - 1 ? pz : 0);

    const S *fin = static_cast<const S *>(a.fin);
    float f[Q];
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        f[q] = ld<S>(fin + (size_t)q * a.P + src[PL::dir(q)]);
        if (kScaled) f[q] *= a.scale[q];
    }
    const float inv_eps = __ldg(a.inv_eps + c);

    // TF/SF: only cells within one cell of the total-field box surface.
    if (a.tfsf) {
        const bool near = x >= a.tf_lo[0] - 1 && x <= a.tf_hi[0] + 1 && y >= a.tf_lo[1] - 1 &&
                          y <= a.tf_hi[1] + 1 && z >= a.tf_lo[2] - 1 && z <= a.tf_hi[2] + 1;
        if (near) {
            const bool in_r = in_box(x, y, z, a.tf_lo, a.tf_hi);
#pragma unroll
            for (int i = 1; i < 7; ++i) {
                const int d = dir_axis(i), sg = dir_sign(i);
                int sx = x, sy = y, sz = z;
                if (d == 0) sx = min(max(x - sg, 0), a.nx - 1);
                if (d == 1) sy = min(max(y - sg, 0), a.ny - 1);
                if (d == 2) sz = min(max(z - sg, 0), a.nz - 1);
                const bool in_s = in_box(sx, sy, sz, a.tf_lo, a.tf_hi);
                if (in_r != in_s) {
                    const float sign = in_r ? 1.f : -1.f;
                    const int sa = a.inc_axis == 0 ? sx : (a.inc_axis == 1 ? sy : sz);
#pragma unroll
                    for (int q = 0; q < Q; ++q)
                        if (PL::dir(q) == i) f[q] += sign * a.inc[(size_t)q * a.n_line + sa];
                }
            }
        }
    }

    float D[3], E[3], H[3];
    moments<MODE>(f, inv_eps, D, E, H);

    if (a.dft_on && in_box(x, y, z, a.nt_lo, a.nt_hi)) {
        const int g[3] = {x, y, z};
        const int n3[3] = {a.nx, a.ny, a.nz};
        float vals[PL::NC];
#pragma unroll
        for (int k = 0; k < PL::NE; ++k) vals[k] = E[Mode<MODE>::ec(k)];
#pragma unroll
        for (int k = 0; k < PL::NH; ++k) vals[PL::NE + k] = H[Mode<MODE>::hc(k)];
        int face = 0;
        for (int ax = 0; ax < 3; ++ax) {
            if (n3[ax] <= 1) continue;
            for (int side = 0; side < 2; ++side, ++face) {
                if (g[ax] != (side ? a.nt_hi[ax] : a.nt_lo[ax])) continue;
                const int ua = ax == 2 ? 1 : 2, va = ax == 0 ? 1 : 0;
                const int iu = g[ua] - a.nt_lo[ua], iv = g[va] - a.nt_lo[va];
                const int nu = a.face_nu[face], nv = a.face_nv[face];
                double *base = a.dft + a.face_off[face] + (long long)iu * nv + iv;
                const long long plane = (long long)nu * nv;
#pragma unroll
                for (int k = 0; k < PL::NC; ++k) {
                    const double v = a.dft_scale * (double)vals[k];
                    base[(2 * k + 0) * plane] += v * a.dft_c;
                    base[(2 * k + 1) * plane] -= v * a.dft_s;
                }
            }
        }
    }

    collide<MODE>(f, D, E, H);

    int d = min(x, a.nx - 1 - x);
    d = min(d, min(y, a.ny - 1 - y));
    if (a.nz > 1) d = min(d, min(z, a.nz - 1 - z));
    const float keep = layer_keep(d, a.w, a.sigma_max, a.inv_w);

    S *fout = static_cast<S *>(a.fout);
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        float v = f[q] * keep;
        if (kScaled) v *= a.inv_scale[q];
        st<S>(fout + (size_t)q * a.P + c, v);
    }
}

constexpr int kBX = 128;

template <int MODE, class S>
cudaError_t launch_t(const StepArgs &a, cudaStream_t s)
{
    const int nblk = a.nblk_main + (a.line_on ? 1 : 0);
    step_kernel<MODE, S, kBX><<<nblk, kBX, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace

int step_block_x() { return kBX; }

cudaError_t launch_step(int mode, int storage, const StepArgs &a, cudaStream_t s)
{
    switch (mode * 3 + storage) {
    case 0: return launch_t<0, float>(a, s);
    case 1: return launch_t<0, __half>(a, s);
    case 2: return launch_t<0, __nv_bfloat16>(a, s);
    case 3: return launch_t<1, float>(a, s);
    case 4: return launch_t<1, __half>(a, s);
    case 5: return launch_t<1, __nv_bfloat16>(a, s);
    case 6: return launch_t<2, float>(a, s);
    case 7: return launch_t<2, __half>(a, s);
    case 8: return launch_t<2, __nv_bfloat16>(a, s);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace lbem
