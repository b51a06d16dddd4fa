// Device code of one lattice-site update shared by the single-step kernels
// (step.cu) and the two-step passes (step2.cu): moments, collision with the
// incident source and the absorbing layer, the running DFT of the NTFF faces,
// the incident line, and the grouped population loads and stores.  Internal
// to liblbem (internal linkage in each translation unit that includes it).
#pragma once

#include <cuda.h>

#include <algorithm>
#include <cstring>
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

}  // namespace
}  // namespace lbem
