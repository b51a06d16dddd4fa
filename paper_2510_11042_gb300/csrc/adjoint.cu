// Discrete adjoint of the fused step (FP32 populations) and the gradient of a
// weighted sum of far-field intensities, J = sum_k w_k |S(theta_k, phi_k)|^2
// (Sec. 2.3-2.4, Eqs. 5-10), with respect to the relative permittivity of
// every cell.
//
// With beta = 1/eps_r, one forward step of the stored (scattered-field)
// populations is
//     u(t)  = S G*(t-1)                              clamped pull (Eq. 1, 4)
//     G*(t) = K [C_beta u(t) + s_beta(t)]            collision, source, layer
// where s_beta is the incident-field source of dielectric cells inside the
// total-field box.  C_beta u = 2 f_eq(E = beta D, H = B) - u is linear in u,
// and both C_beta u and s_beta depend on beta only through E = beta D^F, D^F
// the total-field D of the pulled populations.  The DFT samples E = beta D,
// H = B of u(t) on the NTFF surface.
//
// The adjoint mu(t) = dJ/du(t) runs backwards:
//     lambda(t) = S^T mu(t+1)                        transposed clamped pull
//     m         = K lambda(t)
//     mu(t)     = C_beta^T m + dJ/du(t)|DFT
// and per cell dJ/dbeta += A . D^F(t), where, with the sums over the moving
// directions i = 1..6 and m_e, m_h the e- and h-components of m,
//     A  = -2 m_e0 + sum_i (m_ei - c_i x m_hi) / 3  + dJ/dE|DFT
//     Bv =           sum_i (m_hi + c_i x m_ei) / 3  + dJ/dH|DFT
// (A is the derivative of m . 2 f_eq with respect to E, Bv with respect to H),
// and C_beta^T m has e_j -> 2 m_e0 + beta A - m_ej, h_j -> Bv - m_hj.  The NTFF
// surface lies outside the total-field box and the absorbing layer, so there
// D^F = D and K = 1.  Finally dJ/deps_r = -beta^2 dJ/dbeta.
//
// S^T as a gather: cell x receives mu_i from x + c_i when that cell exists,
// and its own mu_i where the clamp maps x - c_i back onto x (x on the face
// that c_i points away from).  The gradient term of a step is formed in FP32
// (A and D^F are FP32) and summed over the steps in FP64.
#include <algorithm>

#include "lbem_internal.cuh"

namespace lbem {
namespace {

constexpr int kAdjBX = 128;

// The adjoint populations use the forward state's FP32 grouped layout
// (pop_index): per direction, pairs of values per cell (and a single in 2D),
// each group starting at plane slot i * NC + s0, so a group is one float2 load.
__device__ __forceinline__ float2 ld_pair(const float *p, int k)
{
    return __ldg(reinterpret_cast<const float2 *>(p) + k);
}

template <int MODE>
__global__ void __launch_bounds__(kAdjBX, MODE == 2 ? 7 : 1) adjoint_step_kernel(const AdjointArgs a)
{
    using PL = Planes<MODE>;
    using M = Mode<MODE>;
    constexpr int Q = PL::Q;
    const int b = blockIdx.x;
    const int bx = b % a.nblk_x;
    const int row = b / a.nblk_x;
    const int y = row % a.ny, z = row / a.ny;
    const int x = bx * kAdjBX + threadIdx.x;
    if (x >= a.nx) return;
    const int pz = a.ny * a.nxp;
    const int c = z * pz + y * a.nxp + x;

    // transposed pull of direction i: neighbour x + c_i and / or x itself
    int nb[7];
    bool has_nb[7], self[7];
    nb[0] = c; has_nb[0] = true; self[0] = false;
    nb[1] = c + 1;   has_nb[1] = x < a.nx - 1; self[1] = x == 0;
    nb[2] = c - 1;   has_nb[2] = x > 0;        self[2] = x == a.nx - 1;
    nb[3] = c + a.nxp; has_nb[3] = y < a.ny - 1; self[3] = y == 0;
    nb[4] = c - a.nxp; has_nb[4] = y > 0;        self[4] = y == a.ny - 1;
    nb[5] = c + pz;  has_nb[5] = z < a.nz - 1; self[5] = z == 0;
    nb[6] = c - pz;  has_nb[6] = z > 0;        self[6] = z == a.nz - 1;

    int d = min(x, a.nx - 1 - x);
    d = min(d, min(y, a.ny - 1 - y));
    if (a.nz > 1) d = min(d, min(z, a.nz - 1 - z));
    const float keep = layer_keep(d, a.w, a.sigma_max, a.inv_w);

    constexpr int NC = PL::NC;
    float m[Q];
#pragma unroll
    for (int i = 0; i < 7; ++i) {
        const float *const *g = a.lin_q + i * NC;
#pragma unroll
        for (int s0 = 0; s0 + 1 < NC; s0 += 2) {
            float2 v = has_nb[i] ? ld_pair(g[s0], nb[i]) : make_float2(0.f, 0.f);
            if (self[i]) {
                const float2 w = ld_pair(g[s0], c);
                v.x += w.x;
                v.y += w.y;
            }
            m[slot_plane(MODE, i, s0)] = keep * v.x;
            m[slot_plane(MODE, i, s0 + 1)] = keep * v.y;
        }
        if (NC & 1) {
            float v = has_nb[i] ? __ldg(g[NC - 1] + nb[i]) : 0.f;
            if (self[i]) v += __ldg(g[NC - 1] + c);
            m[slot_plane(MODE, i, NC - 1)] = keep * v;
        }
    }
    float me[7][3], mh[7][3];
#pragma unroll
    for (int i = 0; i < 7; ++i)
#pragma unroll
        for (int k = 0; k < 3; ++k) me[i][k] = mh[i][k] = 0.f;
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        if (PL::fam(q) == 0) me[PL::dir(q)][PL::comp(q)] = m[q];
        else mh[PL::dir(q)][PL::comp(q)] = m[q];
    }

    float sE[3] = {0.f, 0.f, 0.f}, sH[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int i = 1; i < 7; ++i)
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            sE[k] += me[i][k] - cross_c(i, mh[i], k);
            sH[k] += mh[i][k] + cross_c(i, me[i], k);
        }
    float A[3], Bv[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        A[k] = third(sE[k]) - 2.f * me[0][k];
        Bv[k] = third(sH[k]);
    }

    if (a.dft_on && in_box(x, y, z, a.nt_lo, a.nt_hi)) {
        // dJ/dx(t) = Re(G (cos - j sin)) * 2/(P T) for every DFT entry of the cell
        const int g[3] = {x, y, z};
        const int n3[3] = {a.nx, a.ny, a.nz};
        double dx[PL::NC];
#pragma unroll
        for (int k = 0; k < PL::NC; ++k) dx[k] = 0.0;
        int face = 0;
        for (int ax = 0; ax < 3; ++ax) {
            if (n3[ax] <= 1) continue;
            for (int side = 0; side < 2; ++side, ++face) {
                if (g[ax] != (side ? a.nt_hi[ax] : a.nt_lo[ax])) continue;
                const int ua = ax == 2 ? 1 : 2, va = ax == 0 ? 1 : 0;
                const int iu = g[ua] - a.nt_lo[ua], iv = g[va] - a.nt_lo[va];
                const int nv = a.face_nv[face];
                const long long plane = (long long)a.face_nu[face] * nv;
                const double *base = a.G + a.face_off[face] + (long long)iu * nv + iv;
#pragma unroll
                for (int k = 0; k < PL::NC; ++k)
                    dx[k] += base[(2 * k) * plane] * a.dft_c + base[(2 * k + 1) * plane] * a.dft_s;
            }
        }
#pragma unroll
        for (int k = 0; k < PL::NE; ++k) A[M::ec(k)] += (float)(a.dft_scale * dx[k]);
#pragma unroll
        for (int k = 0; k < PL::NH; ++k) Bv[M::hc(k)] += (float)(a.dft_scale * dx[PL::NE + k]);
    }

    // this step's term in FP32 (its factors are FP32), the sum over steps in FP64
    float gs = 0.f;
#pragma unroll
    for (int k = 0; k < PL::NE; ++k) gs = fmaf(A[M::ec(k)], __ldg(a.rec + (long long)k * a.P + c), gs);
    a.grad[c] += (double)gs;

    const float beta = __ldg(a.inv_eps + c);
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        const int k = PL::comp(q);
        const float v = PL::fam(q) == 0 ? fmaf(beta, A[k], 2.f * me[0][k]) : Bv[k];
        m[q] = v - m[q];
    }
#pragma unroll
    for (int i = 0; i < 7; ++i) {
        float *const *g = a.lout_q + i * NC;
#pragma unroll
        for (int s0 = 0; s0 + 1 < NC; s0 += 2)
            reinterpret_cast<float2 *>(g[s0])[c] =
                make_float2(m[slot_plane(MODE, i, s0)], m[slot_plane(MODE, i, s0 + 1)]);
        if (NC & 1) g[NC - 1][c] = m[slot_plane(MODE, i, NC - 1)];
    }
}

// dJ/dN and dJ/dL of each angle from N, L (far_field_finalize) and |E_I|:
// dJ = Re(sum_c gN_c dN_c + gL_c dL_c).
__global__ void adjoint_gamma_kernel(const AdjWeightArgs a)
{
    const int ang = blockIdx.x * blockDim.x + threadIdx.x;
    if (ang >= a.n_ang) return;
    const double *v = a.amp + (long long)ang * 12;
    double ei = 0.0;
    const int nodes[2] = {a.center_i0, a.center_i1};
    for (int t = 0; t < 2; ++t) {
        double re = 0.0, im = 0.0;
        for (int c = 0; c < 3; ++c) {
            re += a.pol[c] * a.line_dft[(nodes[t] * 3 + c) * 2 + 0];
            im += a.pol[c] * a.line_dft[(nodes[t] * 3 + c) * 2 + 1];
        }
        ei += 0.5 * sqrt(re * re + im * im);
    }
    const double th = a.theta[ang], k = a.k, wk = a.weights[ang];
    double gN[3][2] = {{0, 0}, {0, 0}, {0, 0}}, gL[3][2] = {{0, 0}, {0, 0}, {0, 0}};
    if (a.mode == 2) {
        const double ph = a.phi[ang];
        const double st = sin(th), ct = cos(th), sp = sin(ph), cp = cos(ph);
        const double tv[3] = {ct * cp, ct * sp, -st}, pv[3] = {-sp, cp, 0.0};
        double a1[2] = {0, 0}, a2[2] = {0, 0};   // N.t + L.p, N.p - L.t
        for (int c = 0; c < 3; ++c)
            for (int r = 0; r < 2; ++r) {
                a1[r] += tv[c] * v[2 * c + r] + pv[c] * v[6 + 2 * c + r];
                a2[r] += pv[c] * v[2 * c + r] - tv[c] * v[6 + 2 * c + r];
            }
        const double f = 2.0 * wk * k * k * k * k / (16.0 * M_PI * M_PI * ei * ei);
        // 2 kappa conj(a1) (t dN + p dL) + 2 kappa conj(a2) (p dN - t dL)
        for (int c = 0; c < 3; ++c) {
            gN[c][0] = f * (a1[0] * tv[c] + a2[0] * pv[c]);
            gN[c][1] = -f * (a1[1] * tv[c] + a2[1] * pv[c]);
            gL[c][0] = f * (a1[0] * pv[c] - a2[0] * tv[c]);
            gL[c][1] = -f * (a1[1] * pv[c] - a2[1] * tv[c]);
        }
    } else {
        const double pv[3] = {-sin(th), cos(th), 0.0};
        const double f = 2.0 * wk * k * k / (8.0 * M_PI * ei * ei);
        double ar = 0.0, ai = 0.0;
        if (a.mode == 0) {          // a = N_z - L.p
            ar = v[4]; ai = v[5];
            for (int c = 0; c < 3; ++c) { ar -= pv[c] * v[6 + 2 * c]; ai -= pv[c] * v[7 + 2 * c]; }
            gN[2][0] = f * ar; gN[2][1] = -f * ai;
            for (int c = 0; c < 3; ++c) { gL[c][0] = -f * ar * pv[c]; gL[c][1] = f * ai * pv[c]; }
        } else {                    // a = N.p + L_z
            ar = v[10]; ai = v[11];
            for (int c = 0; c < 3; ++c) { ar += pv[c] * v[2 * c]; ai += pv[c] * v[2 * c + 1]; }
            for (int c = 0; c < 3; ++c) { gN[c][0] = f * ar * pv[c]; gN[c][1] = -f * ai * pv[c]; }
            gL[2][0] = f * ar; gL[2][1] = -f * ai;
        }
    }
    double *out = a.gamma + (long long)ang * 12;
    for (int c = 0; c < 3; ++c)
        for (int r = 0; r < 2; ++r) {
            out[2 * c + r] = gN[c][r];
            out[6 + 2 * c + r] = gL[c][r];
        }
}

// G of every DFT entry: sum over angles of gamma times the entry's weight,
// phase and current (J = n x H, M = -n x E), in the DFT array layout.
__global__ void adjoint_weights_kernel(const AdjWeightArgs a)
{
    const long long total = a.g.cell_start[a.g.nfaces];
    for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < total;
         j += (long long)gridDim.x * blockDim.x) {
        int f = 0;
        while (f + 1 < a.g.nfaces && j >= a.g.cell_start[f + 1]) ++f;
        const long long jl = j - a.g.cell_start[f];
        const int nu = a.g.nu[f], nv = a.g.nv[f];
        const int iu = (int)(jl / nv), iv = (int)(jl % nv);
        const int ax = a.g.axis[f];
        const int ua = ax == 2 ? 1 : 2, va = ax == 0 ? 1 : 0;
        double w = 1.0;
        if (nu > 1 && (iu == 0 || iu == nu - 1)) w *= 0.5;
        if (nv > 1 && (iv == 0 || iv == nv - 1)) w *= 0.5;
        double pos[3];
        pos[ax] = a.g.side[f] ? a.g.hi[ax] : a.g.lo[ax];
        pos[ua] = a.g.lo[ua] + iu;
        pos[va] = a.g.lo[va] + iv;
        const double sgn = a.g.side[f] ? 1.0 : -1.0;
        const int b1 = (ax + 1) % 3, b2 = (ax + 2) % 3;
        double GE[3][2] = {{0, 0}, {0, 0}, {0, 0}}, GH[3][2] = {{0, 0}, {0, 0}, {0, 0}};
        for (int ang = 0; ang < a.n_ang; ++ang) {
            const double th = a.theta[ang];
            double rh[3];
            if (a.mode == 2) {
                const double ph = a.phi[ang];
                rh[0] = sin(th) * cos(ph);
                rh[1] = sin(th) * sin(ph);
                rh[2] = cos(th);
            } else {
                rh[0] = cos(th);
                rh[1] = sin(th);
                rh[2] = 0.0;
            }
            double sp, cp;
            sincos(a.k * (rh[0] * (pos[0] - a.center[0]) + rh[1] * (pos[1] - a.center[1]) +
                          rh[2] * (pos[2] - a.center[2])),
                   &sp, &cp);
            const double pr = w * cp, pi = w * sp;
            const double *gm = a.gamma + (long long)ang * 12;
            // (g * p) for g = gamma entry
            auto mul = [&](int idx, double s, double out[2]) {
                out[0] += s * (gm[idx] * pr - gm[idx + 1] * pi);
                out[1] += s * (gm[idx] * pi + gm[idx + 1] * pr);
            };
            // N_b1 += -sgn H_b2 p, N_b2 += sgn H_b1 p; L_b1 += sgn E_b2 p, L_b2 += -sgn E_b1 p
            mul(2 * b1, -sgn, GH[b2]);
            mul(2 * b2, sgn, GH[b1]);
            mul(6 + 2 * b1, sgn, GE[b2]);
            mul(6 + 2 * b2, -sgn, GE[b1]);
        }
        double *base = a.G + a.g.off[f] + jl;
        const long long plane = (long long)nu * nv;
        for (int c = 0; c < 3; ++c) {
            const int se = slot_E(a.mode, c), sh = slot_H(a.mode, c);
            if (se >= 0) {
                base[(2 * se) * plane] = GE[c][0];
                base[(2 * se + 1) * plane] = GE[c][1];
            }
            if (sh >= 0) {
                base[(2 * sh) * plane] = GH[c][0];
                base[(2 * sh + 1) * plane] = GH[c][1];
            }
        }
    }
}

// dJ/deps_r = -beta^2 dJ/dbeta, unpadded [nz][ny][nx]
__global__ void adjoint_finalize_kernel(const double *grad, const float *inv_eps, int nx, int ny,
                                        int nz, int nxp, float *out)
{
    const long long n = (long long)nx * ny * nz;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(i % nx);
        const long long r = i / nx;
        const long long c = r * nxp + x;
        const double b = (double)inv_eps[c];
        out[i] = (float)(-b * b * grad[c]);
    }
}

template <int MODE>
cudaError_t launch_adj(AdjointArgs a, cudaStream_t s)
{
    a.nblk_x = (a.nx + kAdjBX - 1) / kAdjBX;
    const long long blocks = (long long)a.nblk_x * a.ny * a.nz;
    if (blocks > 0x7fffffffLL) return cudaErrorInvalidValue;
    adjoint_step_kernel<MODE><<<(unsigned)blocks, kAdjBX, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_adjoint_step(int mode, const AdjointArgs &a, cudaStream_t s)
{
    switch (mode) {
    case 0: return launch_adj<0>(a, s);
    case 1: return launch_adj<1>(a, s);
    case 2: return launch_adj<2>(a, s);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_adjoint_weights(const AdjWeightArgs &a, cudaStream_t s, int *launches)
{
    if (a.n_ang < 1) return cudaErrorInvalidValue;
    adjoint_gamma_kernel<<<(a.n_ang + 127) / 128, 128, 0, s>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const long long total = a.g.cell_start[a.g.nfaces];
    const int blocks = (int)std::min<long long>((total + 255) / 256, 16LL * std::max(1, sm_count()));
    adjoint_weights_kernel<<<blocks > 0 ? blocks : 1, 256, 0, s>>>(a);
    *launches = 2;
    return cudaGetLastError();
}

cudaError_t launch_adjoint_finalize(const double *grad, const float *inv_eps, int nx, int ny, int nz,
                                    int nxp, float *out, cudaStream_t s)
{
    const long long n = (long long)nx * ny * nz;
    const int blocks = (int)std::min<long long>((n + 255) / 256, 16LL * std::max(1, sm_count()));
    adjoint_finalize_kernel<<<blocks > 0 ? blocks : 1, 256, 0, s>>>(grad, inv_eps, nx, ny, nz, nxp, out);
    return cudaGetLastError();
}

}  // namespace lbem
