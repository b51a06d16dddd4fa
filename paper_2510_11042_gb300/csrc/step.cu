// Fused D3Q7 stream-and-collide step for the lattice-Boltzmann Maxwell scheme
// of arXiv 2510.11042, Sec. 2.1 (Eqs. 1-2) with the outer boundary of Eq. 4.
//
// One launch advances every cell by one time step:
//   pull    f_i(r) = f*_i(clamp(r - c_i))           (Eq. 1 streaming + Eq. 4)
//   TF/SF   incident population of the link's source cell added on links that
//           enter the total-field box, removed on links that leave it
//   moments D = sum_i e_i, B = sum_i h_i, E = D / eps_r, H = B / mu_r
//           (mu_r = 1 unless a permeability map is set)
//   DFT     X += x(t) exp(-j w t) on the NTFF box surface (FP64 accumulators)
//   collide f* = 2 f_eq - f (tau = 1/2, equilibria of Eq. 2):
//             e_0* = 2 (eps_r - 1) E - e_0 = 2 (D - E) - e_0
//             e_i* = (E - c_i x H) / 3 - e_i,    h_0* = 2 (B - H) - h_0,
//             h_i* = (H + c_i x E) / 3 - h_i
//           with E/3 and H/3 free of rounding bias, so that the sum of the moving
//           equilibria, 6 (E/3), carries no systematic rounding bias and D, B
//           are conserved to unbiased rounding;
//   layer   f* *= 1 - sigma_max (m / W)^3 near the outer faces
//   store   to the other ping-pong buffer.
//
// Scattered-field storage.  Inside the total-field box the kernel stores
// G = F - I, the total post-collision population minus the incident one of
// the 1D incident line at the same time and coordinate along k; outside the
// box G = F (there the field is the scattered one).  The link-wise TF/SF rule
// (I added on links entering the box, removed on links leaving it) then reads
// F(r) = G(src) + chi(r) I(src) for every pull, and, C_eps being the linear
// collision of a cell,
//     G*(r) = C_eps(G_pulled) + chi(r) [C_eps(I_pulled) - I(r, n+1)].
// Inside the box the line is the vacuum update, I(r, n+1) = C_1(I_pulled), so
// the bracket is (C_eps - C_1)(I_pulled): zero in vacuum cells and, in a
// dielectric cell, the equilibrium of the field dE = E_inc (1/eps_r - 1) with
// no magnetic part (e_0: -2 dE, e_i: dE/3, h_i: c_i x dE/3), where E_inc is
// the line's field at time n+1.  So every cell runs the plain update on G and
// only dielectric cells inside the box add that source.  The stored values are
// scattered fields everywhere, which keeps reduced-precision storage errors
// proportional to the scattered field rather than to the incident one.
//
// The incident line (same update, eps_r = 1, absorbing layer at both ends,
// hard source) runs one step ahead of the lattice in three rotating buffers:
// during step n the lattice reads line(n+1) and the first blocks of the same
// launch write line(n+2).
//
// Memory layout: per velocity direction, the direction's populations in
// groups of 2 (FP32) or 4 and 2 (16-bit, 3D) consecutive values per cell, each
// group a plane-sized array of nz*ny*nxp cells, x fastest and padded to a
// multiple of 32 cells (pop_index in lbem_internal.cuh); 4 B of 1/eps_r per
// cell.  One vector load fetches a group, so a 3D cell takes 21 (FP32) or
// 14 (16-bit) loads.  Each population is read once and written once per
// step: B_cell = 2 Q s + 4 bytes.  The update is a
// memory-bound stencil (~1 flop/byte), so it runs on the CUDA cores; no
// tensor-core path applies.
#include <cuda.h>

#include <algorithm>
#include <cstring>
#include <mutex>
#include <type_traits>

#include "lbem_internal.cuh"

namespace lbem {
namespace {

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

// f <- 2 f_eq - f.  2 e_i^eq = (E - c_i x H)/3 = E/3 - c_i x (H/3) for i != 0.
template <int MODE>
__device__ __forceinline__ void collide(float *f, const float D[3], const float E[3],
                                        const float H[3])
{
    using PL = Planes<MODE>;
    using M = Mode<MODE>;
    float E3[3] = {0.f, 0.f, 0.f}, H3[3] = {0.f, 0.f, 0.f};
    // only the components the mode carries are non-zero
#pragma unroll
    for (int k = 0; k < PL::NE; ++k) E3[M::ec(k)] = third(E[M::ec(k)]);
#pragma unroll
    for (int k = 0; k < PL::NH; ++k) H3[M::hc(k)] = third(H[M::hc(k)]);
#pragma unroll
    for (int q = 0; q < PL::Q; ++q) {
        const int i = PL::dir(q), a = PL::comp(q);
        float eq2;  // 2 f_eq
        if (PL::fam(q) == 0)
            eq2 = (i == 0) ? 2.f * (D[a] - E[a]) : E3[a] - cross_c(i, H3, a);
        else
            eq2 = (i == 0) ? 0.f : H3[a] + cross_c(i, E3, a);
        f[q] = eq2 - f[q];
    }
}

// One node s of the incident line: line_out[.][s] = update of line_in at node s
// (pull along the line with the clamped ends, eps_r = 1 moments and collision,
// absorbing layer at both ends, hard source overwrite at src_index).
template <int MODE>
__device__ __noinline__ void line_node(const float *__restrict__ line_in, float *__restrict__ line_out,
                                       int n, int s, int w, float sigma_max, float inv_w,
                                       int src_index, float sE0, float sE1, float sE2, float sH0,
                                       float sH1, float sH2, int axis)
{
    using PL = Planes<MODE>;
    constexpr int Q = PL::Q;
    float f[Q];
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        const int i = PL::dir(q);
        const int c = (dir_axis(i) == axis) ? dir_sign(i) : 0;
        int src = s - c;
        src = src < 0 ? 0 : (src > n - 1 ? n - 1 : src);
        f[q] = line_in[(size_t)q * n + src];
    }
    float D[3], E[3], H[3];
    moments<MODE>(f, 1.f, D, E, H);
    collide<MODE>(f, D, E, H);
    const float keep = layer_keep(min(s, n - 1 - s), w, sigma_max, inv_w);
#pragma unroll
    for (int q = 0; q < Q; ++q) f[q] *= keep;
    if (s == src_index) {
        // vacuum equilibrium of the prescribed incident fields
        const float sE[3] = {sE0, sE1, sE2}, sH[3] = {sH0, sH1, sH2};
        constexpr float sixth = 1.0f / 6.0f;
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            const int i = PL::dir(q), a = PL::comp(q);
            if (i == 0) f[q] = 0.f;
            else if (PL::fam(q) == 0) f[q] = (sE[a] - cross_c(i, sH, a)) * sixth;
            else f[q] = (sH[a] + cross_c(i, sE, a)) * sixth;
        }
    }
#pragma unroll
    for (int q = 0; q < Q; ++q) line_out[(size_t)q * n + s] = f[q];
}

// Line work done by the first blocks of a step: DFT of the line's fields at
// time n+1 (moments of the stored state, conserved by collision) and the
// update line(n+1) -> line(n+2).
template <int MODE>
__device__ __forceinline__ void line_work(const StepArgs &a, int s)
{
    using PL = Planes<MODE>;
    const int n = a.n_line;
    if (a.dft_on) {
        float E[3] = {0.f, 0.f, 0.f};
#pragma unroll
        for (int q = 0; q < 7 * PL::NE; ++q) E[PL::comp(q)] += a.line_n1[(size_t)q * n + s];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const double v = a.dft_scale * (double)E[c];
            a.line_dft[(s * 3 + c) * 2 + 0] += v * a.dft_c;
            a.line_dft[(s * 3 + c) * 2 + 1] -= v * a.dft_s;
        }
    }
    line_node<MODE>(a.line_n1, a.line_out, n, s, a.w, a.sigma_max, a.inv_w, a.src_index,
                    a.src_E[0], a.src_E[1], a.src_E[2], a.src_H[0], a.src_H[1], a.src_H[2],
                    a.inc_axis);
}

// Analytic TF/SF source of a cell inside the total-field box, in storage
// units: keep * C(I_pulled) - I(r, n+1), where I(p, t) is the vacuum
// equilibrium (Eq. 2) of the closed-form plane wave at cell p and time t, and
// I_pulled takes direction i's populations from the cell the clamped pull
// reads, clamp(r - c_i), at time n.  (Storing G = F - I inside the box, the
// link-wise rule F_pulled = G_pulled + chi(r) I_pulled makes
// G* = keep C(G_pulled) + chi(r) [keep C(I_pulled) - I(r, n+1)].)
// Amplitude E0 ramp(tau) sin(w tau) of the closed-form wave at cell (px, py, pz)
// and time t_s, tau = t_s - 3 k.(p - r0), from the per-axis tables in FP32:
// sin(w tau) = Im(exp(j w t_s) prod_a exp(-j w 3 k_a (p_a - r0_a))).  All
// factors have unit modulus, so the phase carries no growing rounding error;
// tau (only needed during the ramp) is formed from small terms.
__device__ __forceinline__ float2 cmulf(float2 p, float2 q)
{
    return make_float2(p.x * q.x - p.y * q.y, p.x * q.y + p.y * q.x);
}

// f = prod_a exp(-j w 3 k_a (p_a - r0_a)) and dsum = sum_a 3 k_a (p_a - r0_a)
// of a cell, then the amplitude at time t_s (s = 0: t_n, 1: t_n+1).
__device__ __forceinline__ float pw_amp_from(const StepArgs &a, float2 f, float dsum, int s)
{
    const float2 w = a.pw_wt[s];
    const float sn = w.x * f.y + w.y * f.x;
    const float tau = a.pw_t[s] - dsum;
    float ramp = 1.f;
    if (tau <= 0.f) ramp = 0.f;
    else if (tau < a.pw_t_ramp) ramp = 0.5f * (1.f - cospif(tau / a.pw_t_ramp));
    return a.pw_amp * ramp * sn;
}

// In-mode field components: EZ carries E_z, H_x, H_y; HZ E_x, E_y, H_z; 3D all.
template <int MODE> __device__ __forceinline__ constexpr bool in_e(int c)
{
    return MODE == 2 || (MODE == 0 ? c == 2 : c < 2);
}
template <int MODE> __device__ __forceinline__ constexpr bool in_h(int c)
{
    return MODE == 2 || (MODE == 0 ? c < 2 : c == 2);
}

// The analytic source of one cell, reduced to what its populations need.
// Population q of direction i != 0 of the vacuum equilibrium of a wave of
// amplitude u is u P(q), P = (p - c_i x k')/6 (electric) or (k' + c_i x p)/6
// (magnetic), p the polarisation and k' = k x p; the rest populations are 0.
// So keep * (2 f_eq(I_pulled) - I_pulled) - I(r, n+1) is, per population,
// keep * 2 f_eq(q) - b_i P(q) with b_i = keep amp_i + an, and the moments of
// I_pulled are D = (A p - V x k')/6, B = (A k' + V x p)/6 with A = sum amp_i,
// V = sum amp_i c_i.  Everything is prescaled by keep / scale (b by 1 / scale).
template <int MODE> struct AnaTerms {
    float b[7];
    float e3[3], h3[3];   // E/3, H/3 of the pulled incident moments
    float d0[3], b0[3];   // 2 (D - E), 2 (B - H): the rest populations
};

template <int MODE>
__device__ __forceinline__ void analytic_prepare(const StepArgs &a, int x, int y, int z, float inv_eps,
                                                 float inv_mu, float keep, AnaTerms<MODE> &t)
{
    constexpr float sixth = 1.0f / 6.0f;
    // per-axis factors at the clamped coordinates p-1, p, p+1 of the cell: the
    // seven pulled cells differ from the cell in one coordinate, so their
    // phase products share the pair products of the other two axes
    float2 fa[3][3];
    float da[3][3];
    {
        const int n3[3] = {a.nx, a.ny, a.nz}, p3[3] = {x, y, z};
        int base = 0;
#pragma unroll
        for (int ax = 0; ax < 3; ++ax) {
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const int pk = min(max(p3[ax] - 1 + k, 0), n3[ax] - 1);
                fa[ax][k] = __ldg(a.pw_ph + base + pk);
                da[ax][k] = __ldg(a.pw_d + base + pk);
            }
            base += n3[ax];
        }
    }
    const float2 gxy = cmulf(fa[0][1], fa[1][1]), gxz = cmulf(fa[0][1], fa[2][1]),
                 gyz = cmulf(fa[1][1], fa[2][1]);
    const float2 fc = cmulf(gxy, fa[2][1]);
    const float dc = da[0][1] + da[1][1] + da[2][1];
    float amp[7];
#pragma unroll
    for (int i = 1; i < 7; ++i) {
        const int d = dir_axis(i), k = 1 - dir_sign(i);  // the pull reads p - c_i
        const float2 f = d == 0 ? cmulf(fa[0][k], gyz) : (d == 1 ? cmulf(fa[1][k], gxz) : cmulf(fa[2][k], gxy));
        const float dsum = da[0][d == 0 ? k : 1] + da[1][d == 1 ? k : 1] + da[2][d == 2 ? k : 1];
        amp[i] = pw_amp_from(a, f, dsum, 0);
    }
    const float an = pw_amp_from(a, fc, dc, 1);
    const float *pol = a.pw_polf, *kxp = a.pw_kxpf;
    const float A = ((amp[1] + amp[2]) + (amp[3] + amp[4])) + (amp[5] + amp[6]);
    const float V[3] = {amp[1] - amp[2], amp[3] - amp[4], amp[5] - amp[6]};
    const float s = keep * a.inv_scale;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const int c1 = (c + 1) % 3, c2 = (c + 2) % 3;
        const float D = in_e<MODE>(c) ? (A * pol[c] - (V[c1] * kxp[c2] - V[c2] * kxp[c1])) * sixth : 0.f;
        const float B = in_h<MODE>(c) ? (A * kxp[c] + (V[c1] * pol[c2] - V[c2] * pol[c1])) * sixth : 0.f;
        const float E = D * inv_eps, H = B * inv_mu;
        t.e3[c] = s * third(E);
        t.h3[c] = s * third(H);
        t.d0[c] = s * (2.f * (D - E));
        t.b0[c] = s * (2.f * (B - H));
    }
    t.b[0] = 0.f;
#pragma unroll
    for (int i = 1; i < 7; ++i) t.b[i] = (keep * amp[i] + an) * a.inv_scale;
}

template <int MODE>
__device__ __forceinline__ float analytic_term(const StepArgs &a, const AnaTerms<MODE> &t, int q)
{
    using PL = Planes<MODE>;
    constexpr float sixth = 1.0f / 6.0f;
    const int i = PL::dir(q), c = PL::comp(q);
    const float *pol = a.pw_polf, *kxp = a.pw_kxpf;
    if (PL::fam(q) == 0) {
        if (i == 0) return t.d0[c];
        return (t.e3[c] - cross_c(i, t.h3, c)) - t.b[i] * ((pol[c] - cross_c(i, kxp, c)) * sixth);
    }
    if (i == 0) return t.b0[c];
    return (t.h3[c] + cross_c(i, t.e3, c)) - t.b[i] * ((kxp[c] + cross_c(i, pol, c)) * sixth);
}

// Accessor of one cell's pulled populations held in registers.
struct FloatCell {
    float *f;
    __device__ __forceinline__ float get(int q) const { return f[q]; }
    __device__ __forceinline__ void set(int q, float v) { f[q] = v; }
};

// Moments, DFT, collision, incident source and absorbing layer of one cell,
// in one pass over its populations after the moments:
//   f* = (2 f_eq - f + source) * keep.
// Values are in storage units (population / scale); fields go to the DFT
// multiplied back by the scale (dft_scale_cells), the incident source is
// divided by it.
template <int MODE, bool REC = false, bool MU = false, bool ANA = false, bool ALLSTAGE = false, class Cell>
__device__ __forceinline__ void update_cell(Cell &f, int x, int y, int z, float inv_eps,
                                            const StepArgs &a, float inv_mu = 1.0f, bool surface = true)
{
    using PL = Planes<MODE>;
    using M = Mode<MODE>;
    constexpr int Q = PL::Q;
    float D[3] = {0.f, 0.f, 0.f}, B[3] = {0.f, 0.f, 0.f};
    if constexpr (MODE == 2) {
        // the same sums in packed pairs (D_x D_y), (D_z B_x), (B_y B_z): each
        // lane adds in direction order, as the scalar loop below does
        float2 p1 = make_float2(0.f, 0.f), p2 = p1, p3 = p1;
#pragma unroll
        for (int i = 0; i < 7; ++i) {
            p1 = __fadd2_rn(p1, make_float2(f.get(3 * i), f.get(3 * i + 1)));
            p2 = __fadd2_rn(p2, make_float2(f.get(3 * i + 2), f.get(21 + 3 * i)));
            p3 = __fadd2_rn(p3, make_float2(f.get(22 + 3 * i), f.get(23 + 3 * i)));
        }
        D[0] = p1.x;
        D[1] = p1.y;
        D[2] = p2.x;
        B[0] = p2.y;
        B[1] = p3.x;
        B[2] = p3.y;
    } else {
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            if (PL::fam(q) == 0) D[PL::comp(q)] += f.get(q);
            else B[PL::comp(q)] += f.get(q);
        }
    }
    if (REC) {
        // total-field D of this step's pulled populations, for the adjoint's
        // permittivity derivative
        float Dinc[3] = {0.f, 0.f, 0.f};
        if (a.tfsf && in_box(x, y, z, a.tf_lo, a.tf_hi)) {
            const int sl = a.inc_axis == 0 ? x : (a.inc_axis == 1 ? y : z);
#pragma unroll
            for (int q = 0; q < 7 * PL::NE; ++q)
                Dinc[PL::comp(q)] += __ldg(a.line_n1 + (size_t)q * a.n_line + sl);
        }
        const long long c = ((long long)z * a.ny + y) * a.nxp + x;
#pragma unroll
        for (int k = 0; k < PL::NE; ++k)
            a.rec[(long long)k * a.P + c] = D[M::ec(k)] * a.scale + Dinc[M::ec(k)];
    }
    // E = D / eps_r and H = B / mu_r as products rounded on their own
    // (__fmul_rn is never contracted into a later add, so every kernel that
    // inlines this update rounds the fields the same way)
    float E[3], H[3], E3[3] = {0.f, 0.f, 0.f}, H3[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int c3 = 0; c3 < 3; ++c3) {
        E[c3] = __fmul_rn(D[c3], inv_eps);
        H[c3] = MU ? __fmul_rn(B[c3], inv_mu) : B[c3];
    }

    bool on_face = surface && a.dft_on && in_box(x, y, z, a.nt_lo, a.nt_hi);
    if constexpr (ALLSTAGE) {
        // the two-step kernel is issue-bound: keep the cells inside the box out
        // of the face loop
        on_face = on_face && (x == a.nt_lo[0] || x == a.nt_hi[0] || y == a.nt_lo[1] || y == a.nt_hi[1] ||
                              z == a.nt_lo[2] || z == a.nt_hi[2]);
    }
    if (on_face) {
        const int g[3] = {x, y, z};
        const int n3[3] = {a.nx, a.ny, a.nz};
        float vals[PL::NC];
#pragma unroll
        for (int k = 0; k < PL::NE; ++k) vals[k] = E[M::ec(k)];
#pragma unroll
        for (int k = 0; k < PL::NH; ++k) vals[PL::NE + k] = H[M::hc(k)];
        int face = 0;
        for (int ax = 0; ax < 3; ++ax) {
            if (n3[ax] <= 1) continue;
            for (int side = 0; side < 2; ++side, ++face) {
                if (g[ax] != (side ? a.nt_hi[ax] : a.nt_lo[ax])) continue;
                const int ua = ax == 2 ? 1 : 2, va = ax == 0 ? 1 : 0;
                const int iu = g[ua] - a.nt_lo[ua], iv = g[va] - a.nt_lo[va];
                const int nu = a.face_nu[face], nv = a.face_nv[face];
                // Staged faces store the fields and dft_flush_x sums them in full
                // warps (3D only: in 2D the branch cost more than it saved).  The
                // single step stages the x faces, which hold two cells per row, one
                // thread in a warp, whose read-modify-write would hold the warp for
                // a DRAM round trip and a lone FP64 pass; the two-step kernel
                // (ALLSTAGE) stages every face, since there the stall would hold
                // a whole tile at every plane.
                if constexpr (MODE == 2 && ALLSTAGE) {
                    if (a.xstage) {
                        const long long j = a.xs_start[face] + (long long)iu * nv + iv;
#pragma unroll
                        for (int k = 0; k < PL::NC; ++k) a.xstage[(long long)k * a.xs_n + j] = vals[k];
                        continue;
                    }
                } else if constexpr (MODE == 2) {
                    if (ax == 0 && a.xstage) {
                        const long long j = ((long long)side * nu + iu) * nv + iv;
#pragma unroll
                        for (int k = 0; k < PL::NC; ++k) a.xstage[(long long)k * a.xs_n + j] = vals[k];
                        continue;
                    }
                }
                double *base = a.dft + a.face_off[face] + (long long)iu * nv + iv;
                const long long plane = (long long)nu * nv;
#pragma unroll
                for (int k = 0; k < PL::NC; ++k) {
                    const double v = (double)vals[k];
                    base[(2 * k + 0) * plane] = fma(v, a.dft_sc, base[(2 * k + 0) * plane]);
                    base[(2 * k + 1) * plane] = fma(v, -a.dft_ss, base[(2 * k + 1) * plane]);
                }
            }
        }
    }

#pragma unroll
    for (int k = 0; k < PL::NE; ++k) E3[M::ec(k)] = third(E[M::ec(k)]);
#pragma unroll
    for (int k = 0; k < PL::NH; ++k) H3[M::hc(k)] = third(H[M::hc(k)]);

    int d = min(x, a.nx - 1 - x);
    d = min(d, min(y, a.ny - 1 - y));
    if (a.nz > 1) d = min(d, min(z, a.nz - 1 - z));
    const float keep = layer_keep(d, a.w, a.sigma_max, a.inv_w);

    // incident-field source of dielectric cells inside the total-field box
    // (the box lies outside the absorbing layer, so keep == 1 there)
    // (with magnetic media also the field dH = H_inc (1/mu_r - 1))
    const bool source = a.tfsf == 1 && (inv_eps != 1.0f || (MU && inv_mu != 1.0f)) &&
                        in_box(x, y, z, a.tf_lo, a.tf_hi);
    const bool ana = ANA && in_box(x, y, z, a.tf_lo, a.tf_hi);
    if (!source && !ana && keep == 1.0f) {
        // most cells: plain collision, f* = 2 f_eq - f
        if constexpr (MODE == 2) {
            // in packed pairs (e_x e_y), (e_z h_x), (h_y h_z) per direction:
            // 2 f_eq + (-1) f rounds once, as 2 f_eq - f does
            const float2 m1 = make_float2(-1.f, -1.f);
#pragma unroll
            for (int i = 0; i < 7; ++i) {
                float eq[6];
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    eq[k] = (i == 0) ? 2.f * (D[k] - E[k]) : E3[k] - cross_c(i, H3, k);
                    eq[3 + k] = (i == 0) ? (MU ? 2.f * (B[k] - H[k]) : 0.f) : H3[k] + cross_c(i, E3, k);
                }
                const int qe = 3 * i, qh = 21 + 3 * i;
                const float2 r0 = __ffma2_rn(make_float2(f.get(qe), f.get(qe + 1)), m1, make_float2(eq[0], eq[1]));
                const float2 r1 = __ffma2_rn(make_float2(f.get(qe + 2), f.get(qh)), m1, make_float2(eq[2], eq[3]));
                const float2 r2 = __ffma2_rn(make_float2(f.get(qh + 1), f.get(qh + 2)), m1, make_float2(eq[4], eq[5]));
                f.set(qe, r0.x);
                f.set(qe + 1, r0.y);
                f.set(qe + 2, r1.x);
                f.set(qh, r1.y);
                f.set(qh + 1, r2.x);
                f.set(qh + 2, r2.y);
            }
            return;
        }
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            const int i = PL::dir(q), ac = PL::comp(q);
            float eq2;
            if (PL::fam(q) == 0) eq2 = (i == 0) ? 2.f * (D[ac] - E[ac]) : E3[ac] - cross_c(i, H3, ac);
            else eq2 = (i == 0) ? (MU ? 2.f * (B[ac] - H[ac]) : 0.f) : H3[ac] + cross_c(i, E3, ac);
            f.set(q, eq2 - f.get(q));
        }
        return;
    }
    AnaTerms<MODE> at;
    if constexpr (ANA) {
        if (ana) analytic_prepare<MODE>(a, x, y, z, inv_eps, inv_mu, keep, at);
    }
    float dE[3] = {0.f, 0.f, 0.f}, dE3[3] = {0.f, 0.f, 0.f};
    float dH[3] = {0.f, 0.f, 0.f}, dH3[3] = {0.f, 0.f, 0.f};
    if (source) {
        const int sl = a.inc_axis == 0 ? x : (a.inc_axis == 1 ? y : z);
#pragma unroll
        for (int q = 0; q < 7 * PL::NE; ++q)
            dE[PL::comp(q)] += __ldg(a.line_n1 + (size_t)q * a.n_line + sl);
        const float g = (inv_eps - 1.0f) * a.inv_scale;  // to storage units
#pragma unroll
        for (int c3 = 0; c3 < 3; ++c3) {
            dE[c3] *= g;
            dE3[c3] = third(dE[c3]);
        }
        if (MU) {
#pragma unroll
            for (int q = 7 * PL::NE; q < Q; ++q)
                dH[PL::comp(q)] += __ldg(a.line_n1 + (size_t)q * a.n_line + sl);
            const float gh = (inv_mu - 1.0f) * a.inv_scale;
#pragma unroll
            for (int c3 = 0; c3 < 3; ++c3) {
                dH[c3] *= gh;
                dH3[c3] = third(dH[c3]);
            }
        }
    }

#pragma unroll
    for (int q = 0; q < Q; ++q) {
        const int i = PL::dir(q), ac = PL::comp(q);
        float eq2, src;  // 2 f_eq and the incident source
        if (PL::fam(q) == 0) {
            eq2 = (i == 0) ? 2.f * (D[ac] - E[ac]) : E3[ac] - cross_c(i, H3, ac);
            src = (i == 0) ? -2.f * dE[ac] : (MU ? dE3[ac] - cross_c(i, dH3, ac) : dE3[ac]);
        } else {
            eq2 = (i == 0) ? (MU ? 2.f * (B[ac] - H[ac]) : 0.f) : H3[ac] + cross_c(i, E3, ac);
            src = (i == 0) ? (MU ? -2.f * dH[ac] : 0.f)
                           : (MU ? dH3[ac] + cross_c(i, dE3, ac) : cross_c(i, dE3, ac));
        }
        float v = (eq2 - f.get(q) + src) * keep;
        if constexpr (ANA) {
            if (ana) v += analytic_term<MODE>(a, at, q);
        }
        f.set(q, v);
    }
}

// Vector access to one group of a cell's populations (the storage layout is
// described with pop_index): W = 1, 2 or 4 consecutive slots in one load or
// store, converted to or from FP32; 16-bit pairs use the paired conversions.
template <class S> struct Io;
template <> struct Io<float> {
    static __device__ __forceinline__ void ld1(const void *p, int k, float &a)
    {
        a = __ldg(static_cast<const float *>(p) + k);
    }
    static __device__ __forceinline__ void ld2(const void *p, int k, float &a, float &b)
    {
        const float2 v = __ldg(static_cast<const float2 *>(p) + k);
        a = v.x;
        b = v.y;
    }
    static __device__ __forceinline__ void st1(void *p, int k, float a) { static_cast<float *>(p)[k] = a; }
    static __device__ __forceinline__ void st2(void *p, int k, float a, float b)
    {
        static_cast<float2 *>(p)[k] = make_float2(a, b);
    }
};
template <class H, class H2> struct Io16 {
    static __device__ __forceinline__ float2 unpack(unsigned u)
    {
        H2 h;
        memcpy(&h, &u, 4);
        if constexpr (std::is_same<H, __half>::value) return __half22float2(h);
        else return __bfloat1622float2(h);
    }
    static __device__ __forceinline__ unsigned pack(float a, float b)
    {
        H2 h;
        if constexpr (std::is_same<H, __half>::value) h = __floats2half2_rn(a, b);
        else h = __floats2bfloat162_rn(a, b);
        unsigned u;
        memcpy(&u, &h, 4);
        return u;
    }
    static __device__ __forceinline__ void ld1(const void *p, int k, float &a)
    {
        const H v = __ldg(static_cast<const H *>(p) + k);
        if constexpr (std::is_same<H, __half>::value) a = __half2float(v);
        else a = __bfloat162float(v);
    }
    static __device__ __forceinline__ void ld2(const void *p, int k, float &a, float &b)
    {
        const float2 v = unpack(__ldg(static_cast<const unsigned *>(p) + k));
        a = v.x;
        b = v.y;
    }
    static __device__ __forceinline__ void ld4(const void *p, int k, float &a, float &b, float &c, float &d)
    {
        const uint2 u = __ldg(static_cast<const uint2 *>(p) + k);
        const float2 v0 = unpack(u.x), v1 = unpack(u.y);
        a = v0.x;
        b = v0.y;
        c = v1.x;
        d = v1.y;
    }
    static __device__ __forceinline__ void st1(void *p, int k, float a)
    {
        if constexpr (std::is_same<H, __half>::value) static_cast<H *>(p)[k] = __float2half_rn(a);
        else static_cast<H *>(p)[k] = __float2bfloat16_rn(a);
    }
    static __device__ __forceinline__ void st2(void *p, int k, float a, float b)
    {
        static_cast<unsigned *>(p)[k] = pack(a, b);
    }
    static __device__ __forceinline__ void st4(void *p, int k, float a, float b, float c, float d)
    {
        static_cast<uint2 *>(p)[k] = make_uint2(pack(a, b), pack(c, d));
    }
};
template <> struct Io<__half> : Io16<__half, __half2> {};
template <> struct Io<__nv_bfloat16> : Io16<__nv_bfloat16, __nv_bfloat162> {};

// All populations of one cell: direction i's groups read at cell index src[i]
// (load) or written at c (store); f is indexed by population plane.
template <int MODE, class S>
__device__ __forceinline__ void load_cell(const StepArgs &a, const int src[7], float *f)
{
    constexpr int NC = Planes<MODE>::NC;
#define SQ(s) f[slot_plane(MODE, i, s)]
#pragma unroll
    for (int i = 0; i < 7; ++i) {
        const void *const *b = a.fin_q + i * NC;
        if constexpr (NC == 3) {
            Io<S>::ld2(b[0], src[i], SQ(0), SQ(1));
            Io<S>::ld1(b[2], src[i], SQ(2));
        } else if constexpr (sizeof(S) == 4) {
            Io<S>::ld2(b[0], src[i], SQ(0), SQ(1));
            Io<S>::ld2(b[2], src[i], SQ(2), SQ(3));
            Io<S>::ld2(b[4], src[i], SQ(4), SQ(5));
        } else {
            Io<S>::ld4(b[0], src[i], SQ(0), SQ(1), SQ(2), SQ(3));
            Io<S>::ld2(b[4], src[i], SQ(4), SQ(5));
        }
    }
}

template <int MODE, class S>
__device__ __forceinline__ void store_cell(const StepArgs &a, int c, const float *f)
{
    constexpr int NC = Planes<MODE>::NC;
#pragma unroll
    for (int i = 0; i < 7; ++i) {
        void *const *b = a.fout_q + i * NC;
        if constexpr (NC == 3) {
            Io<S>::st2(b[0], c, SQ(0), SQ(1));
            Io<S>::st1(b[2], c, SQ(2));
        } else if constexpr (sizeof(S) == 4) {
            Io<S>::st2(b[0], c, SQ(0), SQ(1));
            Io<S>::st2(b[2], c, SQ(2), SQ(3));
            Io<S>::st2(b[4], c, SQ(4), SQ(5));
        } else {
            Io<S>::st4(b[0], c, SQ(0), SQ(1), SQ(2), SQ(3));
            Io<S>::st2(b[4], c, SQ(4), SQ(5));
        }
    }
#undef SQ
}

// One thread per cell.  The input group of direction i starts at
// a.fin_q[i * NC + s0] (kernel parameters), so every access is a 32-bit
// in-group offset from a constant-bank base; the +-x pulls are plain loads
// shifted by one element (coalesced; the extra sector per warp hits in L1/L2).
// The cells x = bx * BX + threadIdx.x of row (y, z) for one step.
template <int MODE, class S, int BX, bool REC = false, bool MU = false, bool ANA = false>
__device__ __forceinline__ void row_cells(const StepArgs &a, int bx, int y, int z)
{
    using PL = Planes<MODE>;
    constexpr int Q = PL::Q;
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

    float f[Q];
    load_cell<MODE, S>(a, src, f);
    FloatCell cell{f};
    update_cell<MODE, REC, MU, ANA>(cell, x, y, z, __ldg(a.inv_eps + c), a,
                                    MU ? __ldg(a.inv_mu + c) : 1.0f);
    store_cell<MODE, S>(a, c, f);
}

// One block per tile of BX cells x R consecutive rows (y fastest, then z);
// the first blocks also update the incident line.  R = rows_of<S> blocks of
// several rows cut the per-block start-up cost of short 128-cell rows; grids
// of under one wave of such blocks (7 per SM) take one row per block
// instead (ONE), so that every SM gets work.  72 registers (7 blocks of 128
// threads per SM) hold a cell without spilling; the 3D kernel with the
// closed-form source (ANA) also holds the source terms and takes 96 (5 blocks:
// 2.83 ms at 384^3, against 3.98 ms spilling at 7).  These were chosen by timing
// the 384^3 sphere and 256^2 to 4096^2 EZ grids on GB300.
template <class S> __host__ __device__ constexpr int rows_of() { return sizeof(S) == 4 ? 2 : 4; }

template <int MODE, class S, int BX, bool REC = false, bool MU = false, bool ANA = false, bool ONE = false>
__global__ void __launch_bounds__(BX, (ANA && MODE == 2) ? 5 : 7) step_kernel_cell(const StepArgs a)
{
    constexpr int R = ONE ? 1 : rows_of<S>();
    const int b = blockIdx.x;
    if (a.line_on) {
        const int s = b * BX + threadIdx.x;
        if (s < a.n_line) line_work<MODE>(a, s);
    }
    const int bx = b % a.nblk_x;
    const int r0 = (b / a.nblk_x) * R;
    const int r1 = min(r0 + R, a.ny * a.nz);
    for (int r = r0; r < r1; ++r) row_cells<MODE, S, BX, REC, MU, ANA>(a, bx, r % a.ny, r / a.ny);
}

constexpr int kBX = 128;  // threads per block = cells per row tile

// ---------------------------------------------------------------------------
// Batched persistent kernel: many problems (same mode and storage, any sizes,
// wavelengths and step counts) advance together in one cooperative launch.
// Each global step, the resident blocks stride over a flat list of work items
// (tiles of kBX cells x rows_per_item rows of one problem); a block copies its
// problem's arguments to shared memory and fills in the per-step ones (buffer
// parity, incident-line buffers, hard-source fields at t+2, DFT phase at t+1)
// before running the same row update as the single-problem kernel.  Problems
// that have taken their steps drop out.  Steps are separated by a grid
// barrier whose wait is bounded: a block that gives up sets status bit 1 and
// the kernel stops.
constexpr long long kBarrierPolls = 1LL << 22;   // ~1 s of 256 ns sleeps

__device__ bool grid_barrier(const BatchArgs &b, unsigned nblocks)
{
    __shared__ int give_up;
    __syncthreads();
    if (threadIdx.x == 0) {
        give_up = 0;
        volatile unsigned *gen = b.bar_gen;
        const unsigned g = *gen;
        __threadfence();
        if (atomicAdd(b.bar_count, 1u) == nblocks - 1) {
            *b.bar_count = 0;
            __threadfence();
            atomicAdd(b.bar_gen, 1u);
        } else {
            long long it = 0;
            while (*gen == g) {
                if (++it > kBarrierPolls) {
                    atomicOr(b.status, 2);
                    give_up = 1;
                    break;
                }
                __nanosleep(256);
            }
        }
        __threadfence();
    }
    __syncthreads();
    return give_up == 0;
}

// Per-step arguments of problem P at its time t (state f*(t) -> f*(t+1)).
__device__ void fill_step_args(StepArgs &sa, const BatchProblem &P, long long step, int Q)
{
    const long long t = P.t0 + step;
    const int in = (P.cur0 + (int)(step & 1)) & 1;
    for (int q = 0; q < Q; ++q) {
        sa.fin_q[q] = P.f_base[in] + q * P.plane_bytes;
        sa.fout_q[q] = (void *)(P.f_base[in ^ 1] + q * P.plane_bytes);
    }
    if (!P.has_wave) return;
    sa.line_n1 = P.line[(t + 1) % 3];
    sa.line_out = P.line[(t + 2) % 3];
    // hard source at time t+2: E = E0 ramp(t) sin(w t) p, H = k x E
    const long long ts = t + 2;
    const double tr = (double)ts;
    double ramp = 1.0;
    if (tr <= 0.0) ramp = 0.0;
    else if (tr < P.t_ramp) ramp = 0.5 * (1.0 - cospi(tr / P.t_ramp));
    const double sv = P.amp * ramp * sinpi(2.0 * (double)(ts % P.T) / (double)P.T);
    for (int c = 0; c < 3; ++c) {
        sa.src_E[c] = (float)(sv * P.pol[c]);
        sa.src_H[c] = (float)(sv * P.kxp[c]);
    }
    // DFT of the fields at time t+1
    const long long tf = t + 1;
    sa.dft_on = (P.dft_t0 >= 1 && tf >= P.dft_t0 && tf < P.dft_t0 + (long long)P.dft_periods * P.T);
    if (sa.dft_on) {
        double sp, cp;
        sincospi(2.0 * (double)(tf % P.T) / (double)P.T, &sp, &cp);
        sa.dft_c = cp;
        sa.dft_s = sp;
        sa.dft_scale = 2.0 / ((double)P.dft_periods * P.T);
        sa.dft_scale_cells = sa.dft_scale * P.scale;
        sa.dft_sc = sa.dft_scale_cells * cp;
        sa.dft_ss = sa.dft_scale_cells * sp;
    }
}

template <int MODE, class S>
__global__ void __launch_bounds__(kBX) batch_kernel(const BatchArgs b)
{
    constexpr int Q = Planes<MODE>::Q;
    __shared__ StepArgs sa;        // arguments of (cached_pi, cached_step)
    __shared__ int s_pi;
    int cached_pi = -1;
    long long cached_step = -1;
    for (long long step = 0; step < b.max_steps; ++step) {
        for (int item = blockIdx.x; item < b.nitems; item += gridDim.x) {
            if (threadIdx.x == 0) {
                int lo = 0, hi = b.nprob - 1;
                while (lo < hi) {
                    const int mid = (lo + hi + 1) / 2;
                    if (b.probs[mid].item0 <= item) lo = mid;
                    else hi = mid - 1;
                }
                s_pi = lo;
            }
            __syncthreads();
            const int pi = s_pi;
            const BatchProblem &P = b.probs[pi];
            if (step < P.steps) {  // uniform over the block
                if (pi != cached_pi || step != cached_step) {
                    const int *src = reinterpret_cast<const int *>(&P.a);
                    int *dst = reinterpret_cast<int *>(&sa);
                    for (int i = threadIdx.x; i < (int)(sizeof(StepArgs) / sizeof(int)); i += blockDim.x)
                        dst[i] = src[i];
                    __syncthreads();
                    if (threadIdx.x == 0) fill_step_args(sa, P, step, Q);
                    __syncthreads();
                    cached_pi = pi;
                    cached_step = step;
                }
                const int li = item - P.item0;
                if (sa.line_on) {
                    const int sl = li * kBX + threadIdx.x;
                    if (sl < sa.n_line) line_work<MODE>(sa, sl);
                }
                const int rows = sa.ny * sa.nz;
                const int r0 = (li / sa.nblk_x) * b.rows_per_item;
                const int bx = li % sa.nblk_x;
                for (int r = r0; r < min(r0 + b.rows_per_item, rows); ++r)
                    row_cells<MODE, S, kBX>(sa, bx, r % sa.ny, r / sa.ny);
            }
            __syncthreads();
        }
        if (!grid_barrier(b, gridDim.x)) return;
        if (*((volatile int *)b.status) & 2) return;
    }
}

// First update of a freshly started incident line: line(t+1) from line(t).
template <int MODE>
__global__ void line_init_kernel(const StepArgs a)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s < a.n_line)
        line_node<MODE>(a.line_n, a.line_out, a.n_line, s, a.w, a.sigma_max, a.inv_w, a.src_index,
                        a.src_E[0], a.src_E[1], a.src_E[2], a.src_H[0], a.src_H[1], a.src_H[2],
                        a.inc_axis);
}



// ---------------------------------------------------------------------------
// Two steps per pass over HBM (3D, plain update; FP32, FP16 and BF16 storage):
// temporal blocking in the 2.5D form, level n staged by the tensor-memory
// accelerator (TMA).
//
// A block owns an xy tile of 32 x 8 cells and marches through a chunk of z
// planes; each tile thread keeps one (x, y) column.  For every plane p:
//   * level n+1 (the state after the first step) of the tile and of its four
//     edge halos (one cell beyond each side, no corners: D3Q7 pulls along one
//     axis at a time) is computed from a bundle of level-n boxes in shared
//     memory: the rest, +-x and +-y groups of plane p, the +z group of plane
//     p-1 and the -z group of plane p+1 (each z index clamped to the grid, the
//     zero-gradient boundary of Eq. 4), all over the tile's 8 rows and one row
//     on either side (the +y box one row lower, the -y box one row higher),
//     and 1/eps_r of plane p;
//   * level n+2 of plane p-1 is computed from level n+1: the +-x and +-y groups
//     of plane p-1 from shared memory (tile and halo cells), its rest group,
//     the +z group of plane p-2 and the -z group of plane p from the column's
//     own registers, and written to HBM.
// One elected thread copies the bundle of plane p+2 into the buffer plane p
// has just released while the block computes, so loads stay in flight during
// the arithmetic; bundles alternate between two buffers, each with an
// mbarrier that the copies complete.  Level n+1 of the +-x, +-y groups lives in
// three rotating slots, so one block barrier per plane orders everything.
// Level n is read from HBM and level n+2 written once per two steps.  A halo
// cell needs only the group of the direction that points into the tile but
// costs a full update, and records no DFT (the tile owning the cell does).
// Pulls that clamp at the domain edge read the cell's own value, so halo cells
// outside the domain are never read.  Every update is update_cell, and with
// 16-bit storage level n+1 is rounded to the storage type before it is used,
// so the result is bitwise that of two single steps.
namespace t2 {
constexpr int TX = 32;                   // tile width (cells)
constexpr int EPS_X0 = 4, EPS_W = 40;    // 1/eps_r box: 40 cells from x0 - 4 (16-byte aligned)
__host__ __device__ constexpr int pad128(int b) { return (b + 127) / 128 * 128; }
constexpr long long kWaitNs = 1000000000LL;  // a bounded wait gives up after 1 s
}  // namespace t2

// Tile geometry: 32 x TY cells, its edge halos, the threads (one per tile or
// halo cell, whole warps) and the box rows (the tile's and one on each side).
template <int TY_> struct T2Tile {
    static constexpr int TX = t2::TX, TY = TY_;
    static constexpr int NT = TX * TY;                       // tile cells
    static constexpr int NHALO = 2 * TY + 2 * TX;            // edge-halo cells
    static constexpr int THREADS = (NT + NHALO + 31) / 32 * 32;
    // the thread that issues the copies: an idle lane of the last warp, else
    // the last halo thread
    static constexpr int ISSUER = NT + NHALO < THREADS ? NT + NHALO : THREADS - 1;
    static constexpr int ROWS = TY + 2;
    static constexpr int EPS_BYTES = ROWS * t2::EPS_W * 4;
};

// Shared-memory layout per storage type.  A bundle holds one box per
// direction and 1/eps_r; a slot holds level n+1 of the +-x, +-y groups of the
// tile cells and the one group of each halo cell.
template <class S> struct T2L : T2Tile<16> {
    // 16-bit: tiles of 32 x 16 cells (one block of 608 threads per SM), per
    // direction a quad (8 B) and a pair (4 B) per cell, boxes of 40 cells from
    // x0 - 4 (a 4-byte pair's x coordinate must be a multiple of 4)
    static constexpr int X0 = 4, W = 40;
    static constexpr int QUAD_BYTES = ROWS * W * 8, PAIR_BYTES = ROWS * W * 4;
    static constexpr int PAIR_OFF = t2::pad128(QUAD_BYTES);
    static constexpr int DIR_BYTES = t2::pad128(PAIR_OFF + PAIR_BYTES);
    static constexpr int EPS_OFF = 7 * DIR_BYTES;
    static constexpr int BUNDLE = t2::pad128(EPS_OFF + EPS_BYTES);
    static constexpr unsigned TX_BYTES = 7 * (QUAD_BYTES + PAIR_BYTES) + EPS_BYTES;
    static constexpr int S_TQ = 0, S_TP = 4 * NT * 8, S_HQ = S_TP + 4 * NT * 4, S_HP = S_HQ + NHALO * 8;
    static constexpr int SLOT = S_HP + NHALO * 4;
    static constexpr int SMEM = 2 * BUNDLE + 3 * SLOT;
    static constexpr int MIN_BLOCKS = 1;
    static constexpr int CLUSTER_X = 1;
};
template <> struct T2L<float> : T2Tile<8> {
    // FP32: tiles of 32 x 8 cells (one block of 352 threads per SM), per
    // direction three float2 groups, boxes of 36 cells from x0 - 2
    static constexpr int X0 = 2, W = 36;
    static constexpr int GROUP_BYTES = ROWS * W * 8;
    static constexpr int DIR_BYTES = t2::pad128(3 * GROUP_BYTES);
    static constexpr int EPS_OFF = 7 * DIR_BYTES;
    static constexpr int BUNDLE = t2::pad128(EPS_OFF + EPS_BYTES);
    static constexpr unsigned TX_BYTES = 7 * 3 * GROUP_BYTES + EPS_BYTES;
    static constexpr int S_TILE = 4 * 3 * NT * 8;  // float2 [4 dirs][3][NT], then halo float2 [3][NHALO]
    static constexpr int SLOT = S_TILE + 3 * NHALO * 8;
    static constexpr int SMEM = 2 * BUNDLE + 3 * SLOT;
    static constexpr int MIN_BLOCKS = 1;
    // launched in clusters of two x-adjacent tiles, with the boxes' L2 fetch
    // granularity left at the default (measured at 384^3: 1.93 -> 1.71 ms per
    // update with the evict-first stores); 16-bit storage measured faster
    // without clusters and with 256-byte L2 promotion
    static constexpr int CLUSTER_X = 2;
};
static_assert(T2L<float>::SMEM <= 232448 - 1024, "two-step FP32 shared memory");
static_assert(T2L<__half>::SMEM <= 232448 - 1024, "two-step 16-bit shared memory");

// The six values of one direction of a cell in storage form.
template <class S> struct DirVal { uint2 q; unsigned p; };   // 16-bit: quad + pair
template <> struct DirVal<float> { float2 g[3]; };

template <class S>
__device__ __forceinline__ DirVal<S> to_dir(const float *f, int d)
{
    DirVal<S> v;
    if constexpr (sizeof(S) == 4) {
#pragma unroll
        for (int k = 0; k < 3; ++k) v.g[k] = make_float2(f[slot_plane(2, d, 2 * k)], f[slot_plane(2, d, 2 * k + 1)]);
    } else {
        using IO = Io<S>;
        v.q = make_uint2(IO::pack(f[slot_plane(2, d, 0)], f[slot_plane(2, d, 1)]),
                         IO::pack(f[slot_plane(2, d, 2)], f[slot_plane(2, d, 3)]));
        v.p = IO::pack(f[slot_plane(2, d, 4)], f[slot_plane(2, d, 5)]);
    }
    return v;
}

template <class S>
__device__ __forceinline__ void from_dir(const DirVal<S> &v, float *f, int d)
{
    if constexpr (sizeof(S) == 4) {
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            f[slot_plane(2, d, 2 * k)] = v.g[k].x;
            f[slot_plane(2, d, 2 * k + 1)] = v.g[k].y;
        }
    } else {
        using IO = Io<S>;
        const float2 a = IO::unpack(v.q.x), b = IO::unpack(v.q.y), c = IO::unpack(v.p);
        f[slot_plane(2, d, 0)] = a.x;
        f[slot_plane(2, d, 1)] = a.y;
        f[slot_plane(2, d, 2)] = b.x;
        f[slot_plane(2, d, 3)] = b.y;
        f[slot_plane(2, d, 4)] = c.x;
        f[slot_plane(2, d, 5)] = c.y;
    }
}

// Direction d of the cell at box column col, row row of a bundle.
template <class S>
__device__ __forceinline__ DirVal<S> bundle_get(const unsigned char *buf, int d, int col, int row)
{
    using L = T2L<S>;
    const unsigned char *b = buf + d * L::DIR_BYTES;
    const int i = row * L::W + col;
    DirVal<S> v;
    if constexpr (sizeof(S) == 4) {
#pragma unroll
        for (int k = 0; k < 3; ++k) v.g[k] = reinterpret_cast<const float2 *>(b + k * L::GROUP_BYTES)[i];
    } else {
        v.q = reinterpret_cast<const uint2 *>(b)[i];
        v.p = reinterpret_cast<const unsigned *>(b + L::PAIR_OFF)[i];
    }
    return v;
}

// The pulled populations of the cell (x, y) at box column col, row row: the
// clamped pull of Eqs. 1 and 4 in box coordinates (the +y box starts one row
// higher, the -y box one row lower than the others).
template <class S>
__device__ __forceinline__ void bundle_cell(const unsigned char *buf, int col, int row, int x, int y, int nx,
                                            int ny, float *f)
{
    from_dir<S>(bundle_get<S>(buf, 0, col, row), f, 0);
    from_dir<S>(bundle_get<S>(buf, 1, x > 0 ? col - 1 : col, row), f, 1);
    from_dir<S>(bundle_get<S>(buf, 2, x < nx - 1 ? col + 1 : col, row), f, 2);
    from_dir<S>(bundle_get<S>(buf, 3, col, y > 0 ? row : row + 1), f, 3);
    from_dir<S>(bundle_get<S>(buf, 4, col, y < ny - 1 ? row : row - 1), f, 4);
    from_dir<S>(bundle_get<S>(buf, 5, col, row), f, 5);
    from_dir<S>(bundle_get<S>(buf, 6, col, row), f, 6);
}

// Slot entries: direction d (1..4) of tile cell i, or the group of halo cell i.
template <class S>
__device__ __forceinline__ void slot_put(unsigned char *slot, bool halo, int d, int i, const DirVal<S> &v)
{
    using L = T2L<S>;
    if constexpr (sizeof(S) == 4) {
        float2 *b = reinterpret_cast<float2 *>(slot) + (halo ? 4 * 3 * L::NT + i : (d - 1) * 3 * L::NT + i);
        const int st = halo ? L::NHALO : L::NT;
#pragma unroll
        for (int k = 0; k < 3; ++k) b[k * st] = v.g[k];
    } else {
        const int j = halo ? i : (d - 1) * L::NT + i;
        reinterpret_cast<uint2 *>(slot + (halo ? L::S_HQ : L::S_TQ))[j] = v.q;
        reinterpret_cast<unsigned *>(slot + (halo ? L::S_HP : L::S_TP))[j] = v.p;
    }
}

template <class S>
__device__ __forceinline__ DirVal<S> slot_get(const unsigned char *slot, bool halo, int d, int i)
{
    using L = T2L<S>;
    DirVal<S> v;
    if constexpr (sizeof(S) == 4) {
        const float2 *b =
            reinterpret_cast<const float2 *>(slot) + (halo ? 4 * 3 * L::NT + i : (d - 1) * 3 * L::NT + i);
        const int st = halo ? L::NHALO : L::NT;
#pragma unroll
        for (int k = 0; k < 3; ++k) v.g[k] = b[k * st];
    } else {
        const int j = halo ? i : (d - 1) * L::NT + i;
        v.q = reinterpret_cast<const uint2 *>(slot + (halo ? L::S_HQ : L::S_TQ))[j];
        v.p = reinterpret_cast<const unsigned *>(slot + (halo ? L::S_HP : L::S_TP))[j];
    }
    return v;
}

// ---- TMA and mbarrier (inline PTX)
__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Wait for phase `parity` of an mbarrier; false if it has not completed
// within t2::kWaitNs.
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity)
{
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    for (;;) {
        if (mbar_try_wait(bar, parity)) return true;
        if (global_ns() - t0 > (unsigned long long)t2::kWaitNs) return false;
    }
}

__device__ __forceinline__ void tma_load_4d(uint32_t dst, const CUtensorMap *map, int c0, int c1, int c2, int c3,
                                            uint32_t bar)
{
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], "
        "[%6];" ::"r"(dst),
        "l"(map), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(bar)
        : "memory");
}

__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap *map, int c0, int c1, int c2, uint32_t bar)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
        "[%5];" ::"r"(dst),
        "l"(map), "r"(c0), "r"(c1), "r"(c2), "r"(bar)
        : "memory");
}

struct Step2Args {
    CUtensorMap map_a;    // FP32: the 21 float2 groups; 16-bit: the 7 quads
    CUtensorMap map_b;    // 16-bit: the 7 pairs
    CUtensorMap map_eps;  // 1/eps_r
    StepArgs s1, s2;      // the two steps: s1 reads level n (fin_q), s2 writes level n+2 (fout_q)
    int zc;               // planes per z chunk (blockIdx.z)
};

// Copy the level-n bundle of plane p into the buffer at dst; the copies
// complete the mbarrier bar.  Every x coordinate is x0 - X0 with x0 a
// multiple of 32, so each box starts on a 16-byte boundary.
template <class S>
__device__ __forceinline__ void t2_issue(const Step2Args &P, uint32_t dst, uint32_t bar, int x0, int y0, int p, int nz)
{
    using L = T2L<S>;
    const int pm = p > 0 ? p - 1 : 0, pp = p < nz - 1 ? p + 1 : nz - 1;
    mbar_expect_tx(bar, L::TX_BYTES);
#pragma unroll
    for (int d = 0; d < 7; ++d) {
        const int yb = d == 3 ? y0 - 2 : (d == 4 ? y0 : y0 - 1);
        const int zb = d == 5 ? pm : (d == 6 ? pp : p);
        if constexpr (sizeof(S) == 4) {
            tma_load_4d(dst + d * L::DIR_BYTES, &P.map_a, 2 * (x0 - L::X0), yb, zb, 3 * d, bar);
        } else {
            tma_load_4d(dst + d * L::DIR_BYTES, &P.map_a, 4 * (x0 - L::X0), yb, zb, d, bar);
            tma_load_4d(dst + d * L::DIR_BYTES + L::PAIR_OFF, &P.map_b, 2 * (x0 - L::X0), yb, zb, d, bar);
        }
    }
    tma_load_3d(dst + L::EPS_OFF, &P.map_eps, x0 - t2::EPS_X0, y0 - 1, p, bar);
}

// Halo cell h of a tile at (x0, y0): its coordinates and the direction whose
// group the tile pulls from it (h < TY: x0-1 (+x), < 2 TY: x0+32 (-x),
// < 2 TY + 32: y0-1 (+y), else y0+TY (-y)).
template <class S>
__device__ __forceinline__ void t2_halo(int h, int x0, int y0, int &x, int &y, int &dir)
{
    constexpr int TX = T2L<S>::TX, TY = T2L<S>::TY;
    if (h < TY) { x = x0 - 1; y = y0 + h; dir = 1; }
    else if (h < 2 * TY) { x = x0 + TX; y = y0 + h - TY; dir = 2; }
    else if (h < 2 * TY + TX) { x = x0 + h - 2 * TY; y = y0 - 1; dir = 3; }
    else { x = x0 + h - 2 * TY - TX; y = y0 + TY; dir = 4; }
}

// Store of level n+2 (3D): as store_cell, with an L2 evict-first policy,
// since nothing reads these lines again in the launch and the boxes of the
// next planes should keep the cache.
__device__ __forceinline__ unsigned long long l2_evict_first()
{
    unsigned long long pol;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}

template <class S>
__device__ __forceinline__ void store_cell_evict_first(const StepArgs &a, int c, const float *f)
{
    const unsigned long long pol = l2_evict_first();
#pragma unroll
    for (int i = 0; i < 7; ++i) {
        void *const *b = a.fout_q + i * 6;
        if constexpr (sizeof(S) == 4) {
#pragma unroll
            for (int k = 0; k < 3; ++k)
                asm volatile("st.global.L2::cache_hint.v2.f32 [%0], {%1, %2}, %3;" ::"l"(
                                 static_cast<float2 *>(b[2 * k]) + c),
                             "f"(f[slot_plane(2, i, 2 * k)]), "f"(f[slot_plane(2, i, 2 * k + 1)]), "l"(pol)
                             : "memory");
        } else {
            using IO = Io<S>;
            asm volatile("st.global.L2::cache_hint.v2.b32 [%0], {%1, %2}, %3;" ::"l"(static_cast<uint2 *>(b[0]) + c),
                         "r"(IO::pack(f[slot_plane(2, i, 0)], f[slot_plane(2, i, 1)])),
                         "r"(IO::pack(f[slot_plane(2, i, 2)], f[slot_plane(2, i, 3)])), "l"(pol)
                         : "memory");
            asm volatile("st.global.L2::cache_hint.b32 [%0], %1, %2;" ::"l"(static_cast<unsigned *>(b[4]) + c),
                         "r"(IO::pack(f[slot_plane(2, i, 4)], f[slot_plane(2, i, 5)])), "l"(pol)
                         : "memory");
        }
    }
}

// Level n+2 of tile cell t at (x, y, z) from level n+1: the +-x, +-y groups
// from the slot of plane z (a neighbour in the tile, a halo cell at the tile
// edge, or the cell itself where the pull clamps at the domain edge), the
// rest, +z and -z groups given.
template <class S>
__device__ __forceinline__ void t2_level2(const StepArgs &s2, const unsigned char *slot, int t, int x, int y, int z,
                                          const DirVal<S> &d0, const DirVal<S> &d5, const DirVal<S> &d6, float ie)
{
    constexpr int TX = T2L<S>::TX, TY = T2L<S>::TY;
    const int nx = s2.nx, ny = s2.ny;
    const int tx = t % TX, ty = t / TX;
    float f[Planes<2>::Q];
    from_dir<S>(d0, f, 0);
    {
        const bool h = x > 0 && tx == 0;
        from_dir<S>(slot_get<S>(slot, h, 1, h ? ty : (x > 0 ? t - 1 : t)), f, 1);
    }
    {
        const bool h = x < nx - 1 && tx == TX - 1;
        from_dir<S>(slot_get<S>(slot, h, 2, h ? TY + ty : (x < nx - 1 ? t + 1 : t)), f, 2);
    }
    {
        const bool h = y > 0 && ty == 0;
        from_dir<S>(slot_get<S>(slot, h, 3, h ? 2 * TY + tx : (y > 0 ? t - TX : t)), f, 3);
    }
    {
        const bool h = y < ny - 1 && ty == TY - 1;
        from_dir<S>(slot_get<S>(slot, h, 4, h ? 2 * TY + TX + tx : (y < ny - 1 ? t + TX : t)), f, 4);
    }
    from_dir<S>(d5, f, 5);
    from_dir<S>(d6, f, 6);
    FloatCell cell{f};
    update_cell<2, false, false, false, true>(cell, x, y, z, ie, s2, 1.0f, true);
    store_cell_evict_first<S>(s2, (z * ny + y) * s2.nxp + x, f);
}

template <class S>
__device__ __forceinline__ void step2_body(const Step2Args &P)
{
    using L = T2L<S>;
    constexpr int TX = L::TX, TY = L::TY, NT = L::NT, NHALO = L::NHALO, ISSUER = L::ISSUER;
    using t2::EPS_W;
    using t2::EPS_X0;
    extern __shared__ __align__(1024) unsigned char t2sm[];
    __shared__ __align__(8) unsigned long long bars[2];
    const StepArgs &s1 = P.s1, &s2 = P.s2;
    const int nx = s1.nx, ny = s1.ny, nz = s1.nz;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const int t = threadIdx.x;
    // z chunk of this block: planes [z0, z1); level n+1 runs over [pa, pb],
    // one plane beyond the chunk on each side inside the grid (recomputed
    // there, not recorded by the DFT)
    const int z0 = blockIdx.z * P.zc, z1 = min(nz, z0 + P.zc);
    const int pa = max(z0 - 1, 0), pb = min(z1, nz - 1);
    const int nl1 = pb - pa + 1;  // >= 2 (nz >= 2)
    const uint32_t bar0 = smem_u32(&bars[0]), buf0 = smem_u32(t2sm);
    unsigned char *slots = t2sm + 2 * L::BUNDLE;

    if (t == ISSUER) {
        mbar_init(bar0, 1);
        mbar_init(bar0 + 8, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    __syncthreads();
    if (t == ISSUER) {
        t2_issue<S>(P, buf0, bar0, x0, y0, pa, nz);
        t2_issue<S>(P, buf0 + L::BUNDLE, bar0 + 8, x0, y0, pa + 1, nz);
    }

    // this thread's cell: a tile cell or an edge-halo cell (or none)
    const bool tile = t < NT;
    int x = -1, y = -1, hd = 0;
    const int h = t - NT;
    if (tile) {
        x = x0 + t % TX;
        y = y0 + t / TX;
    } else if (h < NHALO) {
        t2_halo<S>(h, x0, y0, x, y, hd);
    }
    const bool live = x >= 0 && x < nx && y >= 0 && y < ny;
    const int col = x - x0 + L::X0, row = y - y0 + 1;

    // level n+1 groups of this column kept for the second step
    DirVal<S> d0_prev{}, d5_prev{}, d5_pp{}, d6_cur{};
    float ie_prev = 1.f;
    // A copy that does not arrive within the bounded wait fails the block: it
    // stops waiting, computing and issuing, but keeps every barrier, then
    // reports the failure and waits (bounded) for its copies still in flight.
    bool failed = false;  // uniform over the block after each barrier
    int consumed = 0;     // bundles whose copies have landed
    for (int j = 0; j < nl1; ++j) {
        const int p = pa + j;
        const unsigned char *buf = t2sm + (j & 1) * L::BUNDLE;
        unsigned char *slot = slots + (p % 3) * L::SLOT;
        bool bad = false;
        if (!failed) {
            bad = !mbar_wait_bounded(bar0 + 8 * (j & 1), (j >> 1) & 1);
            if (!bad) consumed = j + 1;
        }
        DirVal<S> d0_cur{}, d5_cur{};
        float ie_cur = 1.f;
        if (live && !failed && !bad) {
            float f[Planes<2>::Q];
            bundle_cell<S>(buf, col, row, x, y, nx, ny, f);
            const float ie = reinterpret_cast<const float *>(buf + L::EPS_OFF)[row * EPS_W + (x - x0 + EPS_X0)];
            FloatCell cell{f};
            update_cell<2, false, false, false, true>(cell, x, y, p, ie, s1, 1.0f, tile && p >= z0 && p < z1);
            if (tile) {
#pragma unroll
                for (int d = 1; d <= 4; ++d) slot_put<S>(slot, false, d, t, to_dir<S>(f, d));
                d0_cur = to_dir<S>(f, 0);
                d5_cur = to_dir<S>(f, 5);
                d6_cur = to_dir<S>(f, 6);
                ie_cur = ie;
            } else {
                // the group pointing into the tile (constant indices keep f in registers)
                const DirVal<S> v = hd == 1 ? to_dir<S>(f, 1)
                                  : hd == 2 ? to_dir<S>(f, 2)
                                  : hd == 3 ? to_dir<S>(f, 3)
                                            : to_dir<S>(f, 4);
                slot_put<S>(slot, true, 0, h, v);
            }
        }
        // level n+1 of plane p is complete and its bundle buffer free
        failed = __syncthreads_or(failed || bad) != 0;
        if (!failed && t == ISSUER && j + 2 < nl1) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            t2_issue<S>(P, buf0 + (j & 1) * L::BUNDLE, bar0 + 8 * (j & 1), x0, y0, p + 2, nz);
        }
        // level n+2 of plane p - 1 (p - 1 < z1 holds, since p <= pb <= z1);
        // at p - 1 == 0 the +z pull clamps to the plane itself
        if (!failed && tile && live && p - 1 >= z0)
            t2_level2<S>(s2, slots + ((p - 1) % 3) * L::SLOT, t, x, y, p - 1, d0_prev,
                         p - 1 == 0 ? d5_prev : d5_pp, d6_cur, ie_prev);
        d5_pp = d5_prev;
        d5_prev = d5_cur;
        d0_prev = d0_cur;
        ie_prev = ie_cur;
    }
    if (failed) {
        if (t == ISSUER) {
            atomicOr(s1.status, 1);
            const int issued = min(consumed + 2, nl1);  // at most two bundles ahead of the last one consumed
            for (int k = consumed; k < issued; ++k) mbar_wait_bounded(bar0 + 8 * (k & 1), (k >> 1) & 1);
        }
        return;
    }
    // the last plane of the grid pulls its -z group from itself (Eq. 4)
    if (z1 == nz && tile && live)
        t2_level2<S>(s2, slots + ((nz - 1) % 3) * L::SLOT, t, x, y, nz - 1, d0_prev, d5_pp, d6_cur, ie_prev);
}

// One block per SM (its shared memory): FP32 352 threads, 16-bit 608.
template <class S>
__global__ void __launch_bounds__(T2L<S>::THREADS, T2L<S>::MIN_BLOCKS) step2_kernel(const __grid_constant__ Step2Args P)
{
    step2_body<S>(P);
}

template <class S> struct Step2Kernel {
    static constexpr auto fn = step2_kernel<S>;
};

// The incident line for both steps of a fused pair, in one block: the line
// work of step n (DFT at n+1, line(n+2)), then of step n+1 (DFT at n+2,
// line(n+3)).
template <int MODE>
__global__ void line2_kernel(const __grid_constant__ StepArgs s1, const __grid_constant__ StepArgs s2)
{
    for (int s = threadIdx.x; s < s1.n_line; s += blockDim.x) line_work<MODE>(s1, s);
    __syncthreads();
    for (int s = threadIdx.x; s < s2.n_line; s += blockDim.x) line_work<MODE>(s2, s);
}

// ---------------------------------------------------------------------------
// Two steps per pass over HBM in 2D (EZ and HZ; FP32, FP16 and BF16
// storage): the temporal blocking above with y as the marching axis.  A
// block owns a strip of 128 cells along x and marches along y through a chunk
// of rows; each strip thread keeps one x column.  For every row r:
//   * level n+1 of the strip and of its two edge-halo cells (x0-1 and x0+128)
//     is computed from a bundle of level-n rows in shared memory: the rest,
//     +-x, +-z groups of row r, the +y group of row r-1 and the -y group of
//     row r+1 (each row index clamped to the grid, Eq. 4), boxes from 4 (FP32)
//     or 8 (16-bit) cells left of the strip to as many right of it, and
//     1/eps_r of row r; the +-z pulls of a 2D grid read the cell itself;
//   * level n+2 of row r-1 is computed from level n+1: the +-x groups from
//     shared memory (strip and halo cells), the rest, +-z groups of row r-1,
//     the +y group of row r-2 and the -y group of row r from the column's own
//     registers, and written to HBM.
// One elected thread keeps the copies of up to three rows ahead in flight
// (four bundle buffers, each with its mbarrier).  Level n+1 of the +-x groups
// lives in three rotating slots, so one block barrier per row orders
// everything.  A chunk recomputes level n+1 of one row on each side (not
// recorded by the DFT).  Every update is update_cell; 16-bit storage rounds
// level n+1 to the storage type, so the result is bitwise that of two single
// steps.
namespace t2d {
constexpr int TXS = 128;                 // strip width (cells)
constexpr int THREADS = 160;             // 128 strip cells, 2 halo cells, idle lanes
constexpr int HALO = TXS, ISSUER = TXS + 2;
constexpr int NB = 4;                    // bundle buffers
__host__ __device__ constexpr int pad16(int b) { return (b + 15) / 16 * 16; }
}  // namespace t2d

// Shared-memory layout: per direction a box of pairs (slots 0, 1 of the
// direction) and a box of singles (slot 2).  FP32: pairs as 8-byte elements,
// boxes of 136 cells from x0 - 4; 16-bit: pairs as 4-byte elements, boxes of
// 144 cells from x0 - 8 (a 2-byte single's x coordinate must be a multiple of
// 8).  A slot holds the +x and -x groups of the strip cells and the group of
// each halo cell.
template <class S> struct T2D {
    static constexpr int X0 = sizeof(S) == 4 ? 4 : 8;
    static constexpr int W = t2d::TXS + 2 * X0;
    static constexpr int PE = 2 * (int)sizeof(S), SE = (int)sizeof(S);  // pair / single bytes
    static constexpr int PAIR_BYTES = W * PE, SINGLE_BYTES = W * SE;
    static constexpr int SINGLE_OFF = t2::pad128(PAIR_BYTES);
    static constexpr int DIR_BYTES = t2::pad128(SINGLE_OFF + SINGLE_BYTES);
    static constexpr int EPS_OFF = 7 * DIR_BYTES;
    static constexpr int EPS_BYTES = W * 4;
    static constexpr int BUNDLE = t2::pad128(EPS_OFF + EPS_BYTES);
    static constexpr unsigned TX_BYTES = 7 * (PAIR_BYTES + SINGLE_BYTES) + EPS_BYTES;
    static constexpr int NSLOT = 2 * t2d::TXS + 2;  // [dir 1 | dir 2] x strip, then the two halo cells
    static constexpr int S_S = t2d::pad16(NSLOT * PE);
    static constexpr int SLOT = t2d::pad16(S_S + NSLOT * SE);
    static constexpr int SMEM = t2d::NB * BUNDLE + 3 * SLOT;
    static constexpr int MIN_BLOCKS = sizeof(S) == 4 ? 3 : 4;
};

// The three values of one direction of a 2D cell in storage form.
template <class S> struct DirVal2 { unsigned p; unsigned short s; };  // 16-bit
template <> struct DirVal2<float> { float2 p; float s; };

template <int MODE, class S>
__device__ __forceinline__ DirVal2<S> to_dir2(const float *f, int d)
{
    DirVal2<S> v;
    const float a = f[slot_plane(MODE, d, 0)], b = f[slot_plane(MODE, d, 1)], c = f[slot_plane(MODE, d, 2)];
    if constexpr (sizeof(S) == 4) {
        v.p = make_float2(a, b);
        v.s = c;
    } else {
        v.p = Io<S>::pack(a, b);
        S h;
        if constexpr (std::is_same<S, __half>::value) h = __float2half_rn(c);
        else h = __float2bfloat16_rn(c);
        memcpy(&v.s, &h, 2);
    }
    return v;
}

template <int MODE, class S>
__device__ __forceinline__ void from_dir2(const DirVal2<S> &v, float *f, int d)
{
    if constexpr (sizeof(S) == 4) {
        f[slot_plane(MODE, d, 0)] = v.p.x;
        f[slot_plane(MODE, d, 1)] = v.p.y;
        f[slot_plane(MODE, d, 2)] = v.s;
    } else {
        const float2 ab = Io<S>::unpack(v.p);
        S h;
        memcpy(&h, &v.s, 2);
        f[slot_plane(MODE, d, 0)] = ab.x;
        f[slot_plane(MODE, d, 1)] = ab.y;
        if constexpr (std::is_same<S, __half>::value) f[slot_plane(MODE, d, 2)] = __half2float(h);
        else f[slot_plane(MODE, d, 2)] = __bfloat162float(h);
    }
}

template <class S>
__device__ __forceinline__ DirVal2<S> bundle2_get(const unsigned char *buf, int d, int col)
{
    using L = T2D<S>;
    const unsigned char *b = buf + d * L::DIR_BYTES;
    DirVal2<S> v;
    if constexpr (sizeof(S) == 4) {
        v.p = reinterpret_cast<const float2 *>(b)[col];
        v.s = reinterpret_cast<const float *>(b + L::SINGLE_OFF)[col];
    } else {
        v.p = reinterpret_cast<const unsigned *>(b)[col];
        v.s = reinterpret_cast<const unsigned short *>(b + L::SINGLE_OFF)[col];
    }
    return v;
}

// Slot entry i: direction 1 of strip cell i (i < 128), direction 2 of strip
// cell i - 128 (i < 256), or the group of halo cell i - 256.
template <class S>
__device__ __forceinline__ void slot2_put(unsigned char *slot, int i, const DirVal2<S> &v)
{
    using L = T2D<S>;
    if constexpr (sizeof(S) == 4) {
        reinterpret_cast<float2 *>(slot)[i] = v.p;
        reinterpret_cast<float *>(slot + L::S_S)[i] = v.s;
    } else {
        reinterpret_cast<unsigned *>(slot)[i] = v.p;
        reinterpret_cast<unsigned short *>(slot + L::S_S)[i] = v.s;
    }
}

template <class S>
__device__ __forceinline__ DirVal2<S> slot2_get(const unsigned char *slot, int i)
{
    using L = T2D<S>;
    DirVal2<S> v;
    if constexpr (sizeof(S) == 4) {
        v.p = reinterpret_cast<const float2 *>(slot)[i];
        v.s = reinterpret_cast<const float *>(slot + L::S_S)[i];
    } else {
        v.p = reinterpret_cast<const unsigned *>(slot)[i];
        v.s = reinterpret_cast<const unsigned short *>(slot + L::S_S)[i];
    }
    return v;
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, int c0, int c1, uint32_t bar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
        "[%4];" ::"r"(dst),
        "l"(map), "r"(c0), "r"(c1), "r"(bar)
        : "memory");
}

// Copy the level-n bundle of row r into the buffer at dst (the copies
// complete the mbarrier bar).  Every x coordinate is x0 - X0 with x0 a
// multiple of 128, so each box starts on a 16-byte boundary.
template <class S>
__device__ __forceinline__ void t2d_issue(const Step2Args &P, uint32_t dst, uint32_t bar, int x0, int r, int ny)
{
    using L = T2D<S>;
    const int rm = r > 0 ? r - 1 : 0, rp = r < ny - 1 ? r + 1 : ny - 1;
    mbar_expect_tx(bar, L::TX_BYTES);
#pragma unroll
    for (int d = 0; d < 7; ++d) {
        const int row = d == 3 ? rm : (d == 4 ? rp : r);
        tma_load_3d(dst + d * L::DIR_BYTES, &P.map_a, x0 - L::X0, row, d, bar);
        tma_load_3d(dst + d * L::DIR_BYTES + L::SINGLE_OFF, &P.map_b, x0 - L::X0, row, d, bar);
    }
    tma_load_2d(dst + L::EPS_OFF, &P.map_eps, x0 - L::X0, r, bar);
}

// Level n+2 of strip cell t at (x, y) from level n+1.
template <int MODE, class S>
__device__ __forceinline__ void t2d_level2(const StepArgs &s2, const unsigned char *slot, int t, int x, int y,
                                           const DirVal2<S> &d0, const DirVal2<S> &d3, const DirVal2<S> &d4,
                                           const DirVal2<S> &d5, const DirVal2<S> &d6, float ie)
{
    constexpr int TXS = t2d::TXS;
    const int nx = s2.nx;
    float f[Planes<MODE>::Q];
    from_dir2<MODE, S>(d0, f, 0);
    // +x from x - 1: the left halo cell at the strip edge, the cell itself at the grid edge
    from_dir2<MODE, S>(slot2_get<S>(slot, x == 0 ? t : (t == 0 ? 2 * TXS : t - 1)), f, 1);
    // -x from x + 1: the right halo cell at the strip edge, the cell itself at the grid edge
    from_dir2<MODE, S>(slot2_get<S>(slot, x == nx - 1 ? TXS + t : (t == TXS - 1 ? 2 * TXS + 1 : TXS + t + 1)), f, 2);
    from_dir2<MODE, S>(d3, f, 3);
    from_dir2<MODE, S>(d4, f, 4);
    from_dir2<MODE, S>(d5, f, 5);
    from_dir2<MODE, S>(d6, f, 6);
    FloatCell cell{f};
    update_cell<MODE, false, false, false, true>(cell, x, y, 0, ie, s2, 1.0f, true);
    store_cell<MODE, S>(s2, y * s2.nxp + x, f);
}

template <int MODE, class S>
__device__ __forceinline__ void step2d_body(const Step2Args &P)
{
    using L = T2D<S>;
    constexpr int TXS = t2d::TXS;
    extern __shared__ __align__(1024) unsigned char t2sm[];
    __shared__ __align__(8) unsigned long long bars[t2d::NB];
    const StepArgs &s1 = P.s1, &s2 = P.s2;
    const int nx = s1.nx, ny = s1.ny;
    const int x0 = blockIdx.x * TXS;
    const int t = threadIdx.x;
    // row chunk [y0, y1); level n+1 runs over [pa, pb]
    const int y0 = blockIdx.y * P.zc, y1 = min(ny, y0 + P.zc);
    const int pa = max(y0 - 1, 0), pb = min(y1, ny - 1);
    const int nl1 = pb - pa + 1;  // >= 2 (ny >= 2)
    const uint32_t bar0 = smem_u32(&bars[0]), buf0 = smem_u32(t2sm);
    unsigned char *slots = t2sm + t2d::NB * L::BUNDLE;

    if (t == t2d::ISSUER) {
        for (int b = 0; b < t2d::NB; ++b) mbar_init(bar0 + 8 * b, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    __syncthreads();
    if (t == t2d::ISSUER)
        for (int j = 0; j < t2d::NB && j < nl1; ++j)
            t2d_issue<S>(P, buf0 + j * L::BUNDLE, bar0 + 8 * j, x0, pa + j, ny);

    // this thread's cell: a strip cell, the left or right halo cell, or none
    const bool strip = t < TXS;
    const int x = strip ? x0 + t : (t == t2d::HALO ? x0 - 1 : (t == t2d::HALO + 1 ? x0 + TXS : -1));
    const bool live = x >= 0 && x < nx;
    const int col = x - x0 + L::X0;

    DirVal2<S> d0_prev{}, d3_prev{}, d3_pp{}, d5_prev{}, d6_prev{}, d4_cur{};
    float ie_prev = 1.f;
    bool failed = false;
    int consumed = 0;
    for (int j = 0; j < nl1; ++j) {
        const int p = pa + j;
        const unsigned char *buf = t2sm + (j % t2d::NB) * L::BUNDLE;
        unsigned char *slot = slots + (p % 3) * L::SLOT;
        bool bad = false;
        if (!failed) {
            bad = !mbar_wait_bounded(bar0 + 8 * (j % t2d::NB), (j / t2d::NB) & 1);
            if (!bad) consumed = j + 1;
        }
        DirVal2<S> d0_cur{}, d3_cur{}, d5_cur{}, d6_cur{};
        float ie_cur = 1.f;
        if (live && !failed && !bad) {
            float f[Planes<MODE>::Q];
            from_dir2<MODE, S>(bundle2_get<S>(buf, 0, col), f, 0);
            from_dir2<MODE, S>(bundle2_get<S>(buf, 1, x > 0 ? col - 1 : col), f, 1);
            from_dir2<MODE, S>(bundle2_get<S>(buf, 2, x < nx - 1 ? col + 1 : col), f, 2);
            from_dir2<MODE, S>(bundle2_get<S>(buf, 3, col), f, 3);
            from_dir2<MODE, S>(bundle2_get<S>(buf, 4, col), f, 4);
            from_dir2<MODE, S>(bundle2_get<S>(buf, 5, col), f, 5);
            from_dir2<MODE, S>(bundle2_get<S>(buf, 6, col), f, 6);
            const float ie = reinterpret_cast<const float *>(buf + L::EPS_OFF)[col];
            FloatCell cell{f};
            update_cell<MODE, false, false, false, true>(cell, x, p, 0, ie, s1, 1.0f, strip && p >= y0 && p < y1);
            if (strip) {
                slot2_put<S>(slot, t, to_dir2<MODE, S>(f, 1));
                slot2_put<S>(slot, TXS + t, to_dir2<MODE, S>(f, 2));
                d0_cur = to_dir2<MODE, S>(f, 0);
                d3_cur = to_dir2<MODE, S>(f, 3);
                d4_cur = to_dir2<MODE, S>(f, 4);
                d5_cur = to_dir2<MODE, S>(f, 5);
                d6_cur = to_dir2<MODE, S>(f, 6);
                ie_cur = ie;
            } else {
                // the left halo cell gives the strip its +x group, the right one its -x group
                slot2_put<S>(slot, 2 * TXS + (t - t2d::HALO),
                             t == t2d::HALO ? to_dir2<MODE, S>(f, 1) : to_dir2<MODE, S>(f, 2));
            }
        }
        // level n+1 of row p is complete and its bundle buffer free
        failed = __syncthreads_or(failed || bad) != 0;
        if (!failed && t == t2d::ISSUER && j + t2d::NB < nl1) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            t2d_issue<S>(P, buf0 + (j % t2d::NB) * L::BUNDLE, bar0 + 8 * (j % t2d::NB), x0, p + t2d::NB, ny);
        }
        // level n+2 of row p - 1; at p - 1 == 0 the +y pull clamps to the row itself
        if (!failed && strip && live && p - 1 >= y0)
            t2d_level2<MODE, S>(s2, slots + ((p - 1) % 3) * L::SLOT, t, x, p - 1, d0_prev,
                                p - 1 == 0 ? d3_prev : d3_pp, d4_cur, d5_prev, d6_prev, ie_prev);
        d3_pp = d3_prev;
        d3_prev = d3_cur;
        d0_prev = d0_cur;
        d5_prev = d5_cur;
        d6_prev = d6_cur;
        ie_prev = ie_cur;
    }
    if (failed) {
        if (t == t2d::ISSUER) {
            atomicOr(s1.status, 1);
            const int issued = min(consumed + t2d::NB, nl1);
            for (int k = consumed; k < issued; ++k)
                mbar_wait_bounded(bar0 + 8 * (k % t2d::NB), (k / t2d::NB) & 1);
        }
        return;
    }
    // the last row of the grid pulls its -y group from itself (Eq. 4)
    if (y1 == ny && strip && live)
        t2d_level2<MODE, S>(s2, slots + ((ny - 1) % 3) * L::SLOT, t, x, ny - 1, d0_prev, d3_pp, d4_cur, d5_prev,
                            d6_prev, ie_prev);
}

template <int MODE, class S>
__global__ void __launch_bounds__(t2d::THREADS, T2D<S>::MIN_BLOCKS) step2d_kernel(const __grid_constant__ Step2Args P)
{
    step2d_body<MODE, S>(P);
}

// Sums cnt staged steps of face fields into the FP64 DFT accumulators in step
// order, with the same fma as the direct path: one thread per (face cell,
// component), reads coalesced along the cells.  Slot s holds the faces in
// mask[s].
__global__ void dft_flush_x_kernel(const DftFlushArgs a)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.n * a.nc) return;
    const long long j = i % a.n;
    const int k = (int)(i / a.n);
    int f = 0;
    while (f + 1 < a.nfaces && j >= a.start[f + 1]) ++f;
    unsigned any = 0;
    for (int s = 0; s < a.cnt; ++s) any |= (a.mask[s] >> f) & 1u;
    if (!any) return;
    const long long r = j - a.start[f];
    double *base = a.dft + a.face_off[f] + r;
    double re = base[(2 * k + 0) * a.plane[f]], im = base[(2 * k + 1) * a.plane[f]];
    for (int s = 0; s < a.cnt; ++s) {
        if (!((a.mask[s] >> f) & 1u)) continue;
        const double v = (double)a.stage[((long long)s * a.nc + k) * a.n + j];
        re = fma(v, a.sc[s], re);
        im = fma(v, -a.ss[s], im);
    }
    base[(2 * k + 0) * a.plane[f]] = re;
    base[(2 * k + 1) * a.plane[f]] = im;
}

template <int MODE, class S, bool REC = false, bool MU = false, bool ANA = false>
cudaError_t launch_cell(StepArgs a, cudaStream_t s)
{
    a.nblk_x = (a.nx + kBX - 1) / kBX;
    a.rows_per_block = rows_of<S>();
    if ((long long)a.nblk_x * a.ny * a.nz / a.rows_per_block < 7LL * std::max(1, sm_count()))
        a.rows_per_block = 1;
    a.nblk_main = a.nblk_x * ((a.ny * a.nz + a.rows_per_block - 1) / a.rows_per_block);
    if (a.line_on && (a.n_line + kBX - 1) / kBX > a.nblk_main) return cudaErrorInvalidValue;
    if (REC && a.rec == nullptr) return cudaErrorInvalidValue;
    if (MU && a.inv_mu == nullptr) return cudaErrorInvalidValue;
    if (ANA != (a.tfsf == 2)) return cudaErrorInvalidValue;
    if (a.rows_per_block == 1)
        step_kernel_cell<MODE, S, kBX, REC, MU, ANA, true><<<a.nblk_main, kBX, 0, s>>>(a);
    else
        step_kernel_cell<MODE, S, kBX, REC, MU, ANA, false><<<a.nblk_main, kBX, 0, s>>>(a);
    return cudaGetLastError();
}

template <int MODE, class S>
cudaError_t launch_batch_t(const BatchArgs &b, int grid, cudaStream_t s)
{
    void *args[] = {const_cast<BatchArgs *>(&b)};
    return cudaLaunchCooperativeKernel((const void *)batch_kernel<MODE, S>, dim3(grid), dim3(kBX), args, 0, s);
}

template <int MODE, class S>
int max_blocks_t()
{
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, batch_kernel<MODE, S>, kBX, 0) != cudaSuccess) return 0;
    return n;
}

// ---- host side of the two-step pass
using EncodeTiledFn = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                   const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// cuTensorMapEncodeTiled from the driver, looked up once (the library links
// the CUDA runtime statically and not the driver library).
EncodeTiledFn encode_tiled()
{
    static std::once_flag once;
    static EncodeTiledFn fn = nullptr;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    });
    return fn;
}

// A tiled tensor map without swizzle or interleave; out-of-range box cells
// read zero (never used: pulls clamp inside the grid).
bool encode_map(CUtensorMap *m, CUtensorMapDataType dt, int rank, const void *base, const cuuint64_t *dims,
                const cuuint64_t *strides, const cuuint32_t *box,
                CUtensorMapL2promotion promo = CU_TENSOR_MAP_L2_PROMOTION_L2_256B)
{
    const EncodeTiledFn fn = encode_tiled();
    if (!fn || (reinterpret_cast<uintptr_t>(base) & 15)) return false;
    const cuuint32_t es[5] = {1, 1, 1, 1, 1};
    return fn(m, dt, (cuuint32_t)rank, const_cast<void *>(base), dims, strides, box, es,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, promo,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <class S> constexpr int storage_slot() { return std::is_same<S, float>::value ? 0 : (std::is_same<S, __half>::value ? 1 : 2); }

// Per device: the two-step kernels' shared-memory opt-in and their resident
// blocks per SM (set up once, under a lock).
std::mutex g_step2_mu;
int g_step2_bps[kMaxDevices][3];

template <class S>
cudaError_t step2_setup(int &blocks_per_sm)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_step2_mu);
    int &bps = g_step2_bps[dev][storage_slot<S>()];
    if (bps == 0) {
        e = cudaFuncSetAttribute(Step2Kernel<S>::fn, cudaFuncAttributeMaxDynamicSharedMemorySize, T2L<S>::SMEM);
        if (e != cudaSuccess) return e;
        int n = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, Step2Kernel<S>::fn, T2L<S>::THREADS, T2L<S>::SMEM);
        if (e != cudaSuccess) return e;
        if (n < 1) return cudaErrorInvalidConfiguration;
        bps = n;
    }
    blocks_per_sm = bps;
    return cudaSuccess;
}

// Whether two-step passes pay on this grid: the tiles times z chunks of at
// least 16 planes fill one wave of resident blocks.  The grid must also hold
// a whole box in x and y.
template <class S>
bool step2_worthwhile_t(int nx, int ny, int nz)
{
    if (nx < 64 || ny < T2L<S>::ROWS || nz < 2) return false;
    int bps = 0;
    if (step2_setup<S>(bps) != cudaSuccess) return false;
    using L = T2L<S>;
    const long long tiles = (long long)((nx + L::TX - 1) / L::TX) * ((ny + L::TY - 1) / L::TY);
    return tiles * std::max(1, nz / 16) >= (long long)std::max(1, sm_count()) * bps;
}

template <class S>
cudaError_t launch_step2_t(const StepArgs &s1, const StepArgs &s2, cudaStream_t s)
{
    using L = T2L<S>;
    if (s1.nx < 64 || s1.ny < L::ROWS || s1.nz < 2 || s1.nxp % 32 || s1.P % 32) return cudaErrorInvalidValue;
    int bps = 0;
    cudaError_t e = step2_setup<S>(bps);
    if (e != cudaSuccess) return e;
    Step2Args P;
    std::memset(&P, 0, sizeof P);
    P.s1 = s1;
    P.s2 = s2;
    const char *f = static_cast<const char *>(s1.fin_q[0]);
    const cuuint64_t nxp = s1.nxp, ny = s1.ny, nz = s1.nz, Pn = (cuuint64_t)s1.P;
    bool ok;
    if constexpr (sizeof(S) == 4) {
        // 21 float2 groups, group g at 2 g P elements
        const cuuint64_t dims[4] = {2 * nxp, ny, nz, 21}, str[3] = {8 * nxp, 8 * nxp * ny, 8 * Pn};
        const cuuint32_t box[4] = {2 * L::W, L::ROWS, 1, 3};
        ok = encode_map(&P.map_a, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, f, dims, str, box,
                        CU_TENSOR_MAP_L2_PROMOTION_NONE);
    } else {
        // direction i: its quads at 6 i P elements, its pairs at (6 i + 4) P
        const cuuint64_t dq[4] = {4 * nxp, ny, nz, 7}, sq[3] = {8 * nxp, 8 * nxp * ny, 12 * Pn};
        const cuuint64_t dp[4] = {2 * nxp, ny, nz, 7}, sp[3] = {4 * nxp, 4 * nxp * ny, 12 * Pn};
        const cuuint32_t bq[4] = {4 * L::W, L::ROWS, 1, 1}, bp[4] = {2 * L::W, L::ROWS, 1, 1};
        ok = encode_map(&P.map_a, CU_TENSOR_MAP_DATA_TYPE_UINT16, 4, f, dq, sq, bq) &&
             encode_map(&P.map_b, CU_TENSOR_MAP_DATA_TYPE_UINT16, 4, f + 8 * Pn, dp, sp, bp);
    }
    {
        const cuuint64_t dims[3] = {nxp, ny, nz}, str[2] = {4 * nxp, 4 * nxp * ny};
        const cuuint32_t box[3] = {t2::EPS_W, L::ROWS, 1};
        ok = ok && encode_map(&P.map_eps, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, s1.inv_eps, dims, str, box);
    }
    if (!ok) return cudaErrorInvalidValue;
    if (s1.line_on) {
        line2_kernel<2><<<1, 512, 0, s>>>(P.s1, P.s2);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    // z chunks of about 40 planes: measured at 384^3, chunks of 8 / 21 / 40 /
    // 96 / 384 planes took 1.96 / 1.71 / 1.65 / 1.77 / 1.97 ms per update in
    // FP32 and 1.19 / 1.05 / 1.02 / 1.06 / 1.20 in FP16 (each chunk recomputes
    // level n+1 of one plane on each side; long chunks lose the wave balance
    // and the locality of the blocks running together).  Grids too small to
    // fill two waves of resident blocks that way take more, shorter chunks.
    const long long tiles = (long long)((s1.nx + L::TX - 1) / L::TX) * ((s1.ny + L::TY - 1) / L::TY);
    const long long cap = (long long)std::max(1, sm_count()) * bps;
    int nzc = std::max(1, (s1.nz + 20) / 40);
    while (tiles * nzc < 2 * cap && (s1.nz + nzc) / (nzc + 1) >= 8) ++nzc;
    int zc = (s1.nz + nzc - 1) / nzc;
    P.zc = zc;
    dim3 grid((s1.nx + L::TX - 1) / L::TX, (s1.ny + L::TY - 1) / L::TY, (s1.nz + zc - 1) / zc);
    if constexpr (L::CLUSTER_X > 1) {
        // clusters of x-adjacent tiles (the grid padded to whole clusters;
        // tiles beyond the grid compute nothing)
        grid.x = (grid.x + L::CLUSTER_X - 1) / L::CLUSTER_X * L::CLUSTER_X;
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = grid;
        cfg.blockDim = dim3(L::THREADS);
        cfg.dynamicSmemBytes = L::SMEM;
        cfg.stream = s;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = L::CLUSTER_X;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        e = cudaLaunchKernelEx(&cfg, Step2Kernel<S>::fn, P);
        if (e != cudaSuccess) return e;
    } else {
        Step2Kernel<S>::fn<<<grid, L::THREADS, L::SMEM, s>>>(P);
    }
    return cudaGetLastError();
}

// ---- host side of the 2D two-step pass
int g_step2d_bps[kMaxDevices][6];

template <int MODE, class S>
cudaError_t step2d_setup(int &blocks_per_sm)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_step2_mu);
    int &bps = g_step2d_bps[dev][MODE * 3 + storage_slot<S>()];
    if (bps == 0) {
        e = cudaFuncSetAttribute(step2d_kernel<MODE, S>, cudaFuncAttributeMaxDynamicSharedMemorySize, T2D<S>::SMEM);
        if (e != cudaSuccess) return e;
        int n = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, step2d_kernel<MODE, S>, t2d::THREADS, T2D<S>::SMEM);
        if (e != cudaSuccess) return e;
        if (n < 1) return cudaErrorInvalidConfiguration;
        bps = n;
    }
    blocks_per_sm = bps;
    return cudaSuccess;
}

// Whether 2D two-step passes pay: the strips times chunks of at least 16 rows
// fill two waves of resident blocks (smaller grids sit in L2, where single
// steps cost no HBM traffic anyway); boxes must fit the row.
template <int MODE, class S>
bool step2d_worthwhile_t(int nx, int ny)
{
    if (nx < 256 || ny < 16) return false;
    int bps = 0;
    if (step2d_setup<MODE, S>(bps) != cudaSuccess) return false;
    const long long strips = (nx + t2d::TXS - 1) / t2d::TXS;
    return strips * std::max(1, ny / 16) >= 2LL * std::max(1, sm_count()) * bps;
}

template <int MODE, class S>
cudaError_t launch_step2d_t(const StepArgs &s1, const StepArgs &s2, cudaStream_t s)
{
    using L = T2D<S>;
    if (s1.nz != 1 || s1.nx < 256 || s1.ny < 16 || s1.nxp % 32 || s1.P % 32) return cudaErrorInvalidValue;
    int bps = 0;
    cudaError_t e = step2d_setup<MODE, S>(bps);
    if (e != cudaSuccess) return e;
    Step2Args P;
    std::memset(&P, 0, sizeof P);
    P.s1 = s1;
    P.s2 = s2;
    const char *f = static_cast<const char *>(s1.fin_q[0]);
    const cuuint64_t nxp = s1.nxp, ny = s1.ny, Pn = (cuuint64_t)s1.P;
    // direction i: its pairs at 3 i P elements, its singles at (3 i + 2) P
    const cuuint64_t dims[3] = {nxp, ny, 7};
    const cuuint64_t sp[2] = {L::PE * nxp, 3 * L::SE * Pn}, ss[2] = {L::SE * nxp, 3 * L::SE * Pn};
    const cuuint32_t box[3] = {L::W, 1, 1};
    bool ok = encode_map(&P.map_a, sizeof(S) == 4 ? CU_TENSOR_MAP_DATA_TYPE_UINT64 : CU_TENSOR_MAP_DATA_TYPE_UINT32,
                         3, f, dims, sp, box) &&
              encode_map(&P.map_b, sizeof(S) == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_UINT16,
                         3, f + 2 * L::SE * Pn, dims, ss, box);
    {
        const cuuint64_t de[2] = {nxp, ny}, se[1] = {4 * nxp};
        const cuuint32_t be[2] = {L::W, 1};
        ok = ok && encode_map(&P.map_eps, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, s1.inv_eps, de, se, be);
    }
    if (!ok) return cudaErrorInvalidValue;
    if (s1.line_on) {
        line2_kernel<MODE><<<1, 512, 0, s>>>(P.s1, P.s2);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    // row chunks as the 3D pass's z chunks: about 40 rows, more and shorter
    // (at least 8 rows) where that would not fill two waves
    const long long strips = (s1.nx + t2d::TXS - 1) / t2d::TXS;
    const long long cap = (long long)std::max(1, sm_count()) * bps;
    int nyc = std::max(1, (s1.ny + 20) / 40);
    while (strips * nyc < 2 * cap && (s1.ny + nyc) / (nyc + 1) >= 8) ++nyc;
    P.zc = (s1.ny + nyc - 1) / nyc;
    const dim3 grid((unsigned)strips, (s1.ny + P.zc - 1) / P.zc, 1);
    step2d_kernel<MODE, S><<<grid, t2d::THREADS, L::SMEM, s>>>(P);
    return cudaGetLastError();
}

}  // namespace

int sm_count()
{
    static std::mutex mu;
    static int cache[kMaxDevices];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return 0;
    std::lock_guard<std::mutex> lock(mu);
    if (cache[dev] == 0) {
        int n = 0;
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
        cache[dev] = n;
    }
    return cache[dev];
}

// Failure-path check of the bounded grid barrier: one block waits for an
// arrival that never comes, gives up after the bounded number of polls, sets
// status bit 1 and returns.
__global__ void barrier_selftest_kernel(const BatchArgs b) { grid_barrier(b, gridDim.x + 1); }

cudaError_t launch_barrier_selftest(const BatchArgs &b, cudaStream_t s)
{
    barrier_selftest_kernel<<<1, kBX, 0, s>>>(b);
    return cudaGetLastError();
}

cudaError_t launch_batch(int mode, int storage, const BatchArgs &b, int grid, cudaStream_t s)
{
    switch (mode * 3 + storage) {
    case 0: return launch_batch_t<0, float>(b, grid, s);
    case 1: return launch_batch_t<0, __half>(b, grid, s);
    case 2: return launch_batch_t<0, __nv_bfloat16>(b, grid, s);
    case 3: return launch_batch_t<1, float>(b, grid, s);
    case 4: return launch_batch_t<1, __half>(b, grid, s);
    case 5: return launch_batch_t<1, __nv_bfloat16>(b, grid, s);
    case 6: return launch_batch_t<2, float>(b, grid, s);
    case 7: return launch_batch_t<2, __half>(b, grid, s);
    case 8: return launch_batch_t<2, __nv_bfloat16>(b, grid, s);
    default: return cudaErrorInvalidValue;
    }
}

int batch_max_blocks_per_sm(int mode, int storage)
{
    switch (mode * 3 + storage) {
    case 0: return max_blocks_t<0, float>();
    case 1: return max_blocks_t<0, __half>();
    case 2: return max_blocks_t<0, __nv_bfloat16>();
    case 3: return max_blocks_t<1, float>();
    case 4: return max_blocks_t<1, __half>();
    case 5: return max_blocks_t<1, __nv_bfloat16>();
    case 6: return max_blocks_t<2, float>();
    case 7: return max_blocks_t<2, __half>();
    case 8: return max_blocks_t<2, __nv_bfloat16>();
    default: return 0;
    }
}

cudaError_t launch_dft_flush_x(const DftFlushArgs &a, cudaStream_t s)
{
    if (a.cnt < 1 || a.cnt > kXStage || a.n <= 0) return cudaErrorInvalidValue;
    const long long total = a.n * a.nc;
    dft_flush_x_kernel<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_step2(int mode, int storage, const StepArgs &s1, const StepArgs &s2, cudaStream_t s)
{
    switch (mode * 3 + storage) {
    case 0: return launch_step2d_t<0, float>(s1, s2, s);
    case 1: return launch_step2d_t<0, __half>(s1, s2, s);
    case 2: return launch_step2d_t<0, __nv_bfloat16>(s1, s2, s);
    case 3: return launch_step2d_t<1, float>(s1, s2, s);
    case 4: return launch_step2d_t<1, __half>(s1, s2, s);
    case 5: return launch_step2d_t<1, __nv_bfloat16>(s1, s2, s);
    case 6: return launch_step2_t<float>(s1, s2, s);
    case 7: return launch_step2_t<__half>(s1, s2, s);
    case 8: return launch_step2_t<__nv_bfloat16>(s1, s2, s);
    default: return cudaErrorInvalidValue;
    }
}

bool step2_worthwhile(int mode, int storage, int nx, int ny, int nz)
{
    switch (mode * 3 + storage) {
    case 0: return step2d_worthwhile_t<0, float>(nx, ny);
    case 1: return step2d_worthwhile_t<0, __half>(nx, ny);
    case 2: return step2d_worthwhile_t<0, __nv_bfloat16>(nx, ny);
    case 3: return step2d_worthwhile_t<1, float>(nx, ny);
    case 4: return step2d_worthwhile_t<1, __half>(nx, ny);
    case 5: return step2d_worthwhile_t<1, __nv_bfloat16>(nx, ny);
    case 6: return step2_worthwhile_t<float>(nx, ny, nz);
    case 7: return step2_worthwhile_t<__half>(nx, ny, nz);
    case 8: return step2_worthwhile_t<__nv_bfloat16>(nx, ny, nz);
    default: return false;
    }
}

cudaError_t launch_step(int mode, int storage, const StepArgs &a, cudaStream_t s)
{
    switch (mode * 3 + storage) {
    case 0: return launch_cell<0, float>(a, s);
    case 1: return launch_cell<0, __half>(a, s);
    case 2: return launch_cell<0, __nv_bfloat16>(a, s);
    case 3: return launch_cell<1, float>(a, s);
    case 4: return launch_cell<1, __half>(a, s);
    case 5: return launch_cell<1, __nv_bfloat16>(a, s);
    case 6: return launch_cell<2, float>(a, s);
    case 7: return launch_cell<2, __half>(a, s);
    case 8: return launch_cell<2, __nv_bfloat16>(a, s);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_step_mu(int mode, int storage, const StepArgs &a, cudaStream_t s)
{
    switch (mode * 3 + storage) {
    case 0: return launch_cell<0, float, false, true>(a, s);
    case 1: return launch_cell<0, __half, false, true>(a, s);
    case 2: return launch_cell<0, __nv_bfloat16, false, true>(a, s);
    case 3: return launch_cell<1, float, false, true>(a, s);
    case 4: return launch_cell<1, __half, false, true>(a, s);
    case 5: return launch_cell<1, __nv_bfloat16, false, true>(a, s);
    case 6: return launch_cell<2, float, false, true>(a, s);
    case 7: return launch_cell<2, __half, false, true>(a, s);
    case 8: return launch_cell<2, __nv_bfloat16, false, true>(a, s);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_step_analytic(int mode, int storage, const StepArgs &a, cudaStream_t s)
{
    switch (mode * 3 + storage) {
    case 0: return launch_cell<0, float, false, true, true>(a, s);
    case 1: return launch_cell<0, __half, false, true, true>(a, s);
    case 2: return launch_cell<0, __nv_bfloat16, false, true, true>(a, s);
    case 3: return launch_cell<1, float, false, true, true>(a, s);
    case 4: return launch_cell<1, __half, false, true, true>(a, s);
    case 5: return launch_cell<1, __nv_bfloat16, false, true, true>(a, s);
    case 6: return launch_cell<2, float, false, true, true>(a, s);
    case 7: return launch_cell<2, __half, false, true, true>(a, s);
    case 8: return launch_cell<2, __nv_bfloat16, false, true, true>(a, s);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_step_record(int mode, const StepArgs &a, cudaStream_t s)
{
    switch (mode) {
    case 0: return launch_cell<0, float, true>(a, s);
    case 1: return launch_cell<1, float, true>(a, s);
    case 2: return launch_cell<2, float, true>(a, s);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_line_init(int mode, const StepArgs &a, cudaStream_t s)
{
    const int blocks = (a.n_line + 127) / 128;
    switch (mode) {
    case 0: line_init_kernel<0><<<blocks, 128, 0, s>>>(a); break;
    case 1: line_init_kernel<1><<<blocks, 128, 0, s>>>(a); break;
    case 2: line_init_kernel<2><<<blocks, 128, 0, s>>>(a); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace lbem
