/*
 * lbem_oracle.c -- plain FP64 CPU reference of the D3Q7 lattice-Boltzmann
 * scheme for Maxwell's equations (Sec. 2.1, Eqs. 1-2; open boundary of
 * Sec. 2.2, Eq. 4).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the checker for the CUDA library:
 * it is loaded by tests/, by __graft_entry__.smoke() and by the CPU-baseline
 * leg of bench.py, and by nothing else.  It shares no code, header, table or
 * constant with the CUDA path under paper_2510_11042_gb300/.
 *
 * Everything is IEEE double, no fast-math, built with -ffp-contract=off so
 * the same source gives the same bits on x86-64 and AArch64.  Loops are the
 * obvious ones; the only parallelism is an OpenMP "parallel for" over cells
 * inside a stage, which does not change any per-cell arithmetic.
 *
 * State layout: f[cell][fam][i][a], cell = (z*ny + y)*nx + x,
 *   fam 0 = electric populations e_i, fam 1 = magnetic populations h_i,
 *   i = 0..6 in the order c0 = 0, +x, -x, +y, -y, +z, -z (Sec. 2.1: D3Q7),
 *   a = vector component x, y, z.
 * So every cell carries 2 x 7 x 3 = 42 doubles, in 2D as well (a 2D problem
 * is an nx x ny x 1 lattice whose z axis has length one; pulling along z then
 * reads the cell itself).
 *
 * One step maps the stored post-collision state f*(n) to f*(n+1):
 *   1. pull streaming, f_i(r) = f*_i(r - c_i), with the outer boundary of
 *      Eq. 4 (incoming population copied from the first interior node), which
 *      for a pull is a clamp of the source coordinate into the box;
 *   2. total-field/scattered-field correction on links that cross the TF box;
 *   3. zeroth moments: D = sum_i e_i, B = sum_i h_i, E = D/eps_r, H = B/mu_r;
 *   4. optional single-frequency DFT of (E, H) at time t = n+1;
 *   5. collision with tau = 1/2 (Eq. 1) towards the equilibria of Eq. 2:
 *      f* = 2 f_eq - f;
 *   6. absorbing layer: f* <- (1 - sigma(r)) f*;
 *   7. optional hard source: one cell's populations are overwritten with the
 *      vacuum equilibrium of a prescribed (E, H) (used by the 1D incident line).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_NQ 42

/* D3Q7 velocities (Sec. 2.1): rest, then +-x, +-y, +-z. */
static const int VEL[7][3] = {
    {0, 0, 0}, {1, 0, 0}, {-1, 0, 0}, {0, 1, 0}, {0, -1, 0}, {0, 0, 1}, {0, 0, -1}};

typedef struct {
    int n[3];          /* local box extent (x, y, z) */
    int origin[3];     /* global coordinate of local cell (0,0,0) */
    int gn[3];         /* global extent; axes with gn == 1 carry no absorbing faces */
    int periodic;      /* 0: clamp (Eq. 4); 1: periodic wrap inside the local box */
    const double *eps; /* relative permittivity per local cell */
    const double *mu;  /* relative permeability per local cell, NULL -> 1 */
    int sponge_w;      /* absorbing-layer width in cells, 0 = none */
    double sigma_max;  /* absorbing-layer strength at the outermost cell */
    /* total-field / scattered-field source */
    int tfsf_kind;     /* 0 none, 1 incident populations from a line table,
                          2 analytic plane wave (oblique incidence) */
    int tf_lo[3], tf_hi[3];   /* TF region, inclusive global cell bounds */
    int inc_axis;             /* kind 1: axis the table is indexed along */
    const double *inc_line;   /* kind 1: [gn[inc_axis]][42] incident f* at time n */
    double k_hat[3], pol[3];  /* kind 2: propagation and E directions */
    double amp, omega, t_ramp;/* kind 2: E0, angular frequency, ramp length */
    double r0[3];             /* kind 2: phase origin of the incident wave */
    /* hard source (incident line) */
    int src_cell;             /* local linear index or -1 */
    double src_E[3], src_H[3];
    /* DFT accumulation */
    int dft_on;
    double dft_cos, dft_sin, dft_scale;
    double *dft_acc;          /* [ncell][6][2]: Ex Ey Ez Hx Hy Hz, (re, im) */
    /* optional field output at t = n+1 (pre-collision moments) */
    double *E_out, *H_out;    /* [ncell][3] each, may be NULL */
    /* optional output of the pulled populations (after streaming and TF/SF,
       before collision), [ncell][42]; used by the adjoint */
    double *u_out;
} orc_params;

static void cross3(const double a[3], const double b[3], double out[3])
{
    out[0] = a[1] * b[2] - a[2] * b[1];
    out[1] = a[2] * b[0] - a[0] * b[2];
    out[2] = a[0] * b[1] - a[1] * b[0];
}

/* Eq. 2: equilibria of both families for fields (E, H) and material (eps, mu).
 * out[fam][i][a] */
void orc_equilibrium(const double E[3], const double H[3], double eps, double mu,
                     double out[ORC_NQ])
{
    for (int i = 0; i < 7; ++i) {
        double c[3] = {(double)VEL[i][0], (double)VEL[i][1], (double)VEL[i][2]};
        double cxH[3], cxE[3];
        cross3(c, H, cxH);
        cross3(c, E, cxE);
        for (int a = 0; a < 3; ++a) {
            double e_eq, h_eq;
            if (i == 0) {
                e_eq = (eps - 1.0) * E[a];
                h_eq = (mu - 1.0) * H[a];
            } else {
                e_eq = (E[a] - cxH[a]) / 6.0;
                h_eq = (H[a] + cxE[a]) / 6.0;
            }
            out[(0 * 7 + i) * 3 + a] = e_eq;
            out[(1 * 7 + i) * 3 + a] = h_eq;
        }
    }
}

/* Zeroth moments (Sec. 2.1): D = sum_i e_i, B = sum_i h_i, E = D/eps, H = B/mu. */
void orc_moments(const double f[ORC_NQ], double eps, double mu, double E[3], double H[3])
{
    for (int a = 0; a < 3; ++a) {
        double D = 0.0, B = 0.0;
        for (int i = 0; i < 7; ++i) {
            D += f[(0 * 7 + i) * 3 + a];
            B += f[(1 * 7 + i) * 3 + a];
        }
        E[a] = D / eps;
        H[a] = B / mu;
    }
}

/* Eq. 1 with tau = 1/2: f* = 2 f_eq(E(f), H(f)) - f, for one cell. */
void orc_collide_cell(const double f[ORC_NQ], double eps, double mu, double out[ORC_NQ])
{
    double E[3], H[3], feq[ORC_NQ];
    orc_moments(f, eps, mu, E, H);
    orc_equilibrium(E, H, eps, mu, feq);
    for (int q = 0; q < ORC_NQ; ++q) out[q] = 2.0 * feq[q] - f[q];
}

/* Absorbing layer: sigma = sigma_max (m/W)^3 with m = W - d, d the distance (in
 * cells) to the nearest absorbing face; zero when d >= W. */
double orc_sigma(const int g[3], const int gn[3], int w, double sigma_max)
{
    if (w <= 0) return 0.0;
    int d = -1;
    for (int a = 0; a < 3; ++a) {
        if (gn[a] <= 1) continue;
        int da = g[a] < gn[a] - 1 - g[a] ? g[a] : gn[a] - 1 - g[a];
        if (d < 0 || da < d) d = da;
    }
    if (d < 0 || d >= w) return 0.0;
    double m = (double)(w - d) / (double)w;
    return sigma_max * m * m * m;
}

static int in_tf(const orc_params *p, const int g[3])
{
    for (int a = 0; a < 3; ++a)
        if (g[a] < p->tf_lo[a] || g[a] > p->tf_hi[a]) return 0;
    return 1;
}

/* Raised-cosine turn-on of the incident wave. */
double orc_ramp(double t, double t_ramp)
{
    if (t <= 0.0) return 0.0;
    if (t >= t_ramp) return 1.0;
    return 0.5 * (1.0 - cos(M_PI * t / t_ramp));
}

/* Incident post-collision population at global cell g, time n (tfsf kinds 1, 2). */
static double incident(const orc_params *p, const int g[3], int64_t n, int q)
{
    if (p->tfsf_kind == 1) {
        int s = g[p->inc_axis];
        return p->inc_line[(size_t)s * ORC_NQ + q];
    }
    /* kind 2: vacuum equilibrium of the analytic plane wave at retarded time */
    double proj = 0.0;
    for (int a = 0; a < 3; ++a) proj += p->k_hat[a] * ((double)g[a] - p->r0[a]);
    double tau = (double)n - 3.0 * proj; /* c = 1/3 (Eq. 3) */
    double s = p->amp * orc_ramp(tau, p->t_ramp) * sin(p->omega * tau);
    double E[3], H[3], kxp[3], feq[ORC_NQ];
    cross3(p->k_hat, p->pol, kxp);
    for (int a = 0; a < 3; ++a) {
        E[a] = s * p->pol[a];
        H[a] = s * kxp[a]; /* vacuum impedance is one in lattice units */
    }
    orc_equilibrium(E, H, 1.0, 1.0, feq);
    return feq[q];
}

static int src_coord(int x, int c, int n, int periodic)
{
    int s = x - c;
    if (periodic) return ((s % n) + n) % n;
    if (s < 0) return 0;
    if (s > n - 1) return n - 1;
    return s;
}

/* One full step f*(n) -> f*(n+1).  fin and fout must not alias. */
int orc_step(const orc_params *p, const double *fin, double *fout, int64_t n)
{
    const int nx = p->n[0], ny = p->n[1], nz = p->n[2];
    const size_t ncell = (size_t)nx * ny * nz;
    double *f = (double *)malloc(ncell * ORC_NQ * sizeof(double));
    if (!f) return -1;

    /* 1. pull streaming with the clamped (Eq. 4) or periodic boundary */
#pragma omp parallel for schedule(static)
    for (long long cell = 0; cell < (long long)ncell; ++cell) {
        int x = (int)(cell % nx), y = (int)((cell / nx) % ny), z = (int)(cell / ((size_t)nx * ny));
        for (int fam = 0; fam < 2; ++fam)
            for (int i = 0; i < 7; ++i) {
                int sx = src_coord(x, VEL[i][0], nx, p->periodic);
                int sy = src_coord(y, VEL[i][1], ny, p->periodic);
                int sz = src_coord(z, VEL[i][2], nz, p->periodic);
                size_t src = ((size_t)sz * ny + sy) * nx + sx;
                for (int a = 0; a < 3; ++a)
                    f[cell * ORC_NQ + (fam * 7 + i) * 3 + a] =
                        fin[src * ORC_NQ + (fam * 7 + i) * 3 + a];
            }
    }

    /* 2. TF/SF: a link from r - c_i to r that enters the TF region carries the
     *    incident population in; one that leaves it carries it out. */
    if (p->tfsf_kind) {
#pragma omp parallel for schedule(static)
        for (long long cell = 0; cell < (long long)ncell; ++cell) {
            int x = (int)(cell % nx), y = (int)((cell / nx) % ny), z = (int)(cell / ((size_t)nx * ny));
            int g[3] = {x + p->origin[0], y + p->origin[1], z + p->origin[2]};
            int in_r = in_tf(p, g);
            for (int i = 1; i < 7; ++i) {
                /* the link's source is the cell the pull actually read */
                int gs[3] = {src_coord(x, VEL[i][0], nx, p->periodic) + p->origin[0],
                             src_coord(y, VEL[i][1], ny, p->periodic) + p->origin[1],
                             src_coord(z, VEL[i][2], nz, p->periodic) + p->origin[2]};
                int in_s = in_tf(p, gs);
                if (in_r == in_s) continue;
                double sign = in_r ? 1.0 : -1.0;
                for (int fam = 0; fam < 2; ++fam)
                    for (int a = 0; a < 3; ++a) {
                        int q = (fam * 7 + i) * 3 + a;
                        f[cell * ORC_NQ + q] += sign * incident(p, gs, n, q);
                    }
            }
        }
    }

    if (p->u_out) memcpy(p->u_out, f, ncell * ORC_NQ * sizeof(double));

    /* 3-6. moments, DFT, collision, absorbing layer */
#pragma omp parallel for schedule(static)
    for (long long cell = 0; cell < (long long)ncell; ++cell) {
        int x = (int)(cell % nx), y = (int)((cell / nx) % ny), z = (int)(cell / ((size_t)nx * ny));
        int g[3] = {x + p->origin[0], y + p->origin[1], z + p->origin[2]};
        double eps = p->eps[cell];
        double mu = p->mu ? p->mu[cell] : 1.0;
        const double *fc = f + cell * ORC_NQ;
        double E[3], H[3];
        orc_moments(fc, eps, mu, E, H);
        if (p->E_out)
            for (int a = 0; a < 3; ++a) p->E_out[cell * 3 + a] = E[a];
        if (p->H_out)
            for (int a = 0; a < 3; ++a) p->H_out[cell * 3 + a] = H[a];
        if (p->dft_on) {
            /* X += scale * x(t) * exp(-j w t) = scale * x * (cos - j sin) */
            double *acc = p->dft_acc + cell * 12;
            for (int a = 0; a < 3; ++a) {
                acc[2 * a + 0] += p->dft_scale * E[a] * p->dft_cos;
                acc[2 * a + 1] -= p->dft_scale * E[a] * p->dft_sin;
                acc[6 + 2 * a + 0] += p->dft_scale * H[a] * p->dft_cos;
                acc[6 + 2 * a + 1] -= p->dft_scale * H[a] * p->dft_sin;
            }
        }
        double feq[ORC_NQ];
        orc_equilibrium(E, H, eps, mu, feq);
        double keep = 1.0 - orc_sigma(g, p->gn, p->sponge_w, p->sigma_max);
        for (int q = 0; q < ORC_NQ; ++q)
            fout[cell * ORC_NQ + q] = keep * (2.0 * feq[q] - fc[q]);
    }

    /* 7. hard source */
    if (p->src_cell >= 0) {
        double feq[ORC_NQ];
        orc_equilibrium(p->src_E, p->src_H, 1.0, 1.0, feq);
        for (int q = 0; q < ORC_NQ; ++q) fout[(size_t)p->src_cell * ORC_NQ + q] = feq[q];
    }
    free(f);
    return 0;
}

/* Physical energy density summed over the box: 1/2 sum (eps |E|^2 + mu |H|^2),
 * with E, H the moments of the stored state (diagnostic only). */
double orc_energy(const int n[3], const double *eps, const double *mu, const double *f)
{
    size_t ncell = (size_t)n[0] * n[1] * n[2];
    double total = 0.0;
    for (size_t cell = 0; cell < ncell; ++cell) {
        double E[3], H[3];
        double e = eps[cell], m = mu ? mu[cell] : 1.0;
        orc_moments(f + cell * ORC_NQ, e, m, E, H);
        for (int a = 0; a < 3; ++a) total += 0.5 * (e * E[a] * E[a] + m * H[a] * H[a]);
    }
    return total;
}

/* ------------------------------------------------------------------------
 * Discrete adjoint of the step (for gradients with respect to eps_r).
 * The step is f(n+1) = K C_eps S f(n) + (terms independent of f), with S the
 * clamped pull, C_eps the per-cell collision and K the absorbing-layer
 * factors, so the adjoint state obeys lambda(n) = S^T C_eps^T K lambda(n+1)
 * (plus the sensitivity of the objective to the fields of step n).
 * ------------------------------------------------------------------------ */

/* C_eps^T applied to one cell's vector: C = 2 F_eq - I with F_eq the linear
 * map f -> f_eq(E(f), H(f)) of Eq. 2 (E = D/eps, H = B/mu); its transpose
 * gathers every output's weight back onto D and B:
 *   a_d = dE/dD * [2 (eps-1) m_e0 + sum_i (m_ei + m_hi x c_i) / 3]   (mu = 1: h_0 term 0)
 *   b_d = dH/dB * [2 (mu-1) m_h0 + sum_i (m_hi - m_ei x c_i) / 3]
 * and (C^T m)_q = a_comp(q) (e-family) or b_comp(q) (h-family) minus m_q.  The
 * dot-product test <C x, y> = <x, C^T y> pins it against orc_collide_cell. */
void orc_collide_adjoint_cell(const double m[ORC_NQ], double eps, double mu, double out[ORC_NQ])
{
    double a[3] = {0, 0, 0}, b[3] = {0, 0, 0};
    for (int i = 0; i < 7; ++i) {
        double c[3] = {(double)VEL[i][0], (double)VEL[i][1], (double)VEL[i][2]};
        const double *me = m + (0 * 7 + i) * 3, *mh = m + (1 * 7 + i) * 3;
        if (i == 0) {
            for (int d = 0; d < 3; ++d) {
                a[d] += 2.0 * (eps - 1.0) * me[d];
                b[d] += 2.0 * (mu - 1.0) * mh[d];
            }
            continue;
        }
        double mhxc[3], mexc[3];
        cross3(mh, c, mhxc);
        cross3(me, c, mexc);
        for (int d = 0; d < 3; ++d) {
            a[d] += (me[d] + mhxc[d]) / 3.0;
            b[d] += (mh[d] - mexc[d]) / 3.0;
        }
    }
    for (int d = 0; d < 3; ++d) {
        a[d] /= eps;   /* E = D / eps */
        b[d] /= mu;    /* H = B / mu  */
    }
    for (int i = 0; i < 7; ++i)
        for (int d = 0; d < 3; ++d) {
            out[(0 * 7 + i) * 3 + d] = a[d] - m[(0 * 7 + i) * 3 + d];
            out[(1 * 7 + i) * 3 + d] = b[d] - m[(1 * 7 + i) * 3 + d];
        }
}

/* d(C_eps f)/d eps for one cell (E = D/eps, dE/deps = -D/eps^2):
 *   e_0: 2 d[(eps-1) E]/deps = 2 D / eps^2,   e_i: -(D / eps^2) / 3,
 *   h_i: -(c_i x D / eps^2) / 3,              h_0: 0. */
void orc_collide_deps_cell(const double f[ORC_NQ], double eps, double out[ORC_NQ])
{
    double D[3] = {0, 0, 0};
    for (int i = 0; i < 7; ++i)
        for (int d = 0; d < 3; ++d) D[d] += f[(0 * 7 + i) * 3 + d];
    double g[3];
    for (int d = 0; d < 3; ++d) g[d] = D[d] / (eps * eps);
    for (int i = 0; i < 7; ++i) {
        double c[3] = {(double)VEL[i][0], (double)VEL[i][1], (double)VEL[i][2]}, cxg[3];
        cross3(c, g, cxg);
        for (int d = 0; d < 3; ++d) {
            out[(0 * 7 + i) * 3 + d] = (i == 0) ? 2.0 * g[d] : -g[d] / 3.0;
            out[(1 * 7 + i) * 3 + d] = (i == 0) ? 0.0 : -cxg[d] / 3.0;
        }
    }
}

/* One adjoint step.  lam_in = lambda(n+1) [ncell][42]; u = the pulled state of
 * forward step n (orc_params.u_out); src (optional) = dJ/du(n) [ncell][42],
 * the objective's sensitivity to the pulled populations of step n; grad
 * accumulates dJ/deps_r per cell.  lam_out = lambda(n) = S^T (C^T K lam_in +
 * src), with S^T the literal scatter of the clamped pull:
 * lam_out_i(clamp(r - c_i)) += nu_i(r). */
int orc_adjoint_step(const orc_params *p, const double *lam_in, const double *u, const double *src,
                     double *lam_out, double *grad)
{
    const int nx = p->n[0], ny = p->n[1], nz = p->n[2];
    const size_t ncell = (size_t)nx * ny * nz;
    double *nu = (double *)malloc(ncell * ORC_NQ * sizeof(double));
    if (!nu) return -1;
#pragma omp parallel for schedule(static)
    for (long long cell = 0; cell < (long long)ncell; ++cell) {
        int x = (int)(cell % nx), y = (int)((cell / nx) % ny), z = (int)(cell / ((size_t)nx * ny));
        int g[3] = {x + p->origin[0], y + p->origin[1], z + p->origin[2]};
        double keep = 1.0 - orc_sigma(g, p->gn, p->sponge_w, p->sigma_max);
        double eps = p->eps[cell], mu = p->mu ? p->mu[cell] : 1.0;
        double m[ORC_NQ], ct[ORC_NQ], dc[ORC_NQ];
        for (int q = 0; q < ORC_NQ; ++q) m[q] = keep * lam_in[cell * ORC_NQ + q];
        orc_collide_adjoint_cell(m, eps, mu, ct);
        orc_collide_deps_cell(u + cell * ORC_NQ, eps, dc);
        double gsum = 0.0;
        for (int q = 0; q < ORC_NQ; ++q) gsum += m[q] * dc[q];
        grad[cell] += gsum;
        for (int q = 0; q < ORC_NQ; ++q)
            nu[cell * ORC_NQ + q] = ct[q] + (src ? src[cell * ORC_NQ + q] : 0.0);
    }
    memset(lam_out, 0, ncell * ORC_NQ * sizeof(double));
    for (size_t cell = 0; cell < ncell; ++cell) {
        int x = (int)(cell % nx), y = (int)((cell / nx) % ny), z = (int)(cell / ((size_t)nx * ny));
        for (int fam = 0; fam < 2; ++fam)
            for (int i = 0; i < 7; ++i) {
                int sx = src_coord(x, VEL[i][0], nx, p->periodic);
                int sy = src_coord(y, VEL[i][1], ny, p->periodic);
                int sz = src_coord(z, VEL[i][2], nz, p->periodic);
                size_t s = ((size_t)sz * ny + sy) * nx + sx;
                for (int a = 0; a < 3; ++a) {
                    int q = (fam * 7 + i) * 3 + a;
                    lam_out[s * ORC_NQ + q] += nu[cell * ORC_NQ + q];
                }
            }
    }
    free(nu);
    return 0;
}

/* The pull alone (no collision), for the dot-product test of the scatter. */
void orc_stream(const orc_params *p, const double *fin, double *fout)
{
    const int nx = p->n[0], ny = p->n[1], nz = p->n[2];
    const size_t ncell = (size_t)nx * ny * nz;
    for (size_t cell = 0; cell < ncell; ++cell) {
        int x = (int)(cell % nx), y = (int)((cell / nx) % ny), z = (int)(cell / ((size_t)nx * ny));
        for (int fam = 0; fam < 2; ++fam)
            for (int i = 0; i < 7; ++i) {
                size_t s = ((size_t)src_coord(z, VEL[i][2], nz, p->periodic) * ny +
                            src_coord(y, VEL[i][1], ny, p->periodic)) * nx +
                           src_coord(x, VEL[i][0], nx, p->periodic);
                for (int a = 0; a < 3; ++a)
                    fout[cell * ORC_NQ + (fam * 7 + i) * 3 + a] = fin[s * ORC_NQ + (fam * 7 + i) * 3 + a];
            }
    }
}

/* The scatter S^T alone (the adjoint of orc_stream). */
void orc_stream_adjoint(const orc_params *p, const double *nu, double *out)
{
    const int nx = p->n[0], ny = p->n[1], nz = p->n[2];
    const size_t ncell = (size_t)nx * ny * nz;
    memset(out, 0, ncell * ORC_NQ * sizeof(double));
    for (size_t cell = 0; cell < ncell; ++cell) {
        int x = (int)(cell % nx), y = (int)((cell / nx) % ny), z = (int)(cell / ((size_t)nx * ny));
        for (int fam = 0; fam < 2; ++fam)
            for (int i = 0; i < 7; ++i) {
                size_t s = ((size_t)src_coord(z, VEL[i][2], nz, p->periodic) * ny +
                            src_coord(y, VEL[i][1], ny, p->periodic)) * nx +
                           src_coord(x, VEL[i][0], nx, p->periodic);
                for (int a = 0; a < 3; ++a)
                    out[s * ORC_NQ + (fam * 7 + i) * 3 + a] += nu[cell * ORC_NQ + (fam * 7 + i) * 3 + a];
            }
    }
}

/* Threads of the OpenMP loops (timing the oracle on one core); no effect
 * without OpenMP.  Does not change any result. */
void orc_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

int orc_abi_version(void) { return 2; }
