// In-place streaming with one population buffer (the AA pattern): the same
// update as the pull step of Sec. 2.1 (stream with the Eq. 4 clamp, moments,
// collide, absorbing layer, TF/SF, DFT), applied to a single buffer by
// alternating two kinds of step, so that the populations take half the memory.
//
// Let P_i(x) be the post-collision populations after a step (what the
// two-buffer scheme keeps in buffer slot i of cell x, the "canonical" state).
//  * Push step (from the canonical state): cell x reads P_i(clamp(x - c_i)) as
//    the pull step does and writes its new P_i(x) into slot opp(i) of cell
//    x + c_i.  Afterwards slot opp(i) of cell y holds P_i(clamp(y - c_i)): the
//    streamed state.
//  * In-place step (from the streamed state): cell x reads direction i from
//    its own slot opp(i), and writes its new P_i(x) into its own slot i: the
//    canonical state again.
// In either step a cell reads and writes the same seven locations (its own
// slots; or, in the push step, slot i of x - c_i for every i, which is slot
// opp(j) of x + c_j for j = opp(i)), each once and the read first, so no
// thread reads a location another thread has written in the same launch.
// Two cases at the grid faces (axes of more than one cell) break that and use
// small face buffers:
//  * a cell whose upstream neighbour x - c_i is outside pulls its own P_i(x)
//    (the clamp); in the push step that slot is overwritten by the neighbour
//    x + c_i, so the in-place step before it also copies P_i(x) of these
//    cells to the face buffer FI_i, which the push step reads instead;
//  * a cell whose downstream neighbour x + c_i is outside keeps P_i(x) in FO_i
//    (nobody streams it, but the canonical state holds it).
// The push step also writes P_i(x) into the cell's own slot opp(i) where
// x - c_i is outside: the clamped value the in-place step pulls.  Along a
// 1-cell axis (z in 2D) both neighbours are the cell itself and no face
// buffer is needed.  Arithmetic and rounding are those of the pull step, so
// both schemes give the same populations bit for bit.
#include <algorithm>
#include <climits>
#include <mutex>

#include "lbem_internal.cuh"
#include "step_cell.cuh"

namespace lbem {
namespace {

// direction i = 1..6 lies on axis (i - 1) / 2, positive for odd i
__host__ __device__ constexpr int aa_axis(int i) { return (i - 1) >> 1; }
__host__ __device__ constexpr bool aa_plus(int i) { return (i & 1) != 0; }

// Face buffers keep the population buffer's grouped layout (see pop_index)
// with the face plane in place of P: the group of width W starting at slot s0
// begins at element s0 * plane and holds face cell k's slot s at
// W * k + (s - s0).  So one vector access reads or writes a direction's group
// from either place, and the choice is a select of base and index, not a
// branch (a branch per direction would make a 16-bit cell wait for each load
// in turn before unpacking it).
__host__ __device__ inline long long aa_face_index(int nc, int elem, long long plane, int s, long long k)
{
    const int s0 = group_first(nc, elem, s), w = group_width(nc, elem, s);
    return s0 * plane + w * k + (s - s0);
}

// The groups of direction i: at cell index k through the group pointers b
// (b[s0]: the group starting at slot s0), or, where face is set, at face cell
// fk of the face buffer fb of fplane cells.
template <int MODE, class S>
__device__ __forceinline__ void aa_load_dir(const void *const *b, int k, const void *fb, int fplane, int fk,
                                            bool face, int i, float *f)
{
    constexpr int NC = Planes<MODE>::NC;
    const S *fs = static_cast<const S *>(fb);
    const int kk = face ? fk : k;
#define GB(s0) (face ? static_cast<const void *>(fs + (long long)(s0) * fplane) : b[s0])
#define SQ(s) f[slot_plane(MODE, i, s)]
    if constexpr (NC == 3) {
        Io<S>::ld2(GB(0), kk, SQ(0), SQ(1));
        Io<S>::ld1(GB(2), kk, SQ(2));
    } else if constexpr (sizeof(S) == 4) {
        Io<S>::ld2(GB(0), kk, SQ(0), SQ(1));
        Io<S>::ld2(GB(2), kk, SQ(2), SQ(3));
        Io<S>::ld2(GB(4), kk, SQ(4), SQ(5));
    } else {
        Io<S>::ld4(GB(0), kk, SQ(0), SQ(1), SQ(2), SQ(3));
        Io<S>::ld2(GB(4), kk, SQ(4), SQ(5));
    }
#undef GB
}

template <int MODE, class S>
__device__ __forceinline__ void aa_store_dir(void *const *b, int k, void *fb, int fplane, int fk, bool face, int i,
                                             const float *f)
{
    constexpr int NC = Planes<MODE>::NC;
    S *fs = static_cast<S *>(fb);
    const int kk = face ? fk : k;
#define GB(s0) (face ? static_cast<void *>(fs + (long long)(s0) * fplane) : b[s0])
    if constexpr (NC == 3) {
        Io<S>::st2(GB(0), kk, SQ(0), SQ(1));
        Io<S>::st1(GB(2), kk, SQ(2));
    } else if constexpr (sizeof(S) == 4) {
        Io<S>::st2(GB(0), kk, SQ(0), SQ(1));
        Io<S>::st2(GB(2), kk, SQ(2), SQ(3));
        Io<S>::st2(GB(4), kk, SQ(4), SQ(5));
    } else {
        Io<S>::st4(GB(0), kk, SQ(0), SQ(1), SQ(2), SQ(3));
        Io<S>::st2(GB(4), kk, SQ(4), SQ(5));
    }
#undef GB
#undef SQ
}

// One row tile of cells for one step of the given kind (0 push, 1 in place).
// The host points the group pointers so that the kernel sees its own slot i
// where the scheme puts direction i: the push step writes direction i through
// fout_q (aimed at slot opp(i)) and the in-place step reads it through fin_q
// (aimed at slot opp(i)).
template <int MODE, class S, int BX, bool MU, bool ANA, int KIND>
__device__ __forceinline__ void aa_row(const StepArgs &a, const AaArgs &g, int bx, int y, int z)
{
    constexpr int Q = Planes<MODE>::Q;
    const int x = bx * BX + threadIdx.x;
    if (x >= a.nx) return;
    const int pz = a.ny * a.nxp;
    const int c = z * pz + y * a.nxp + x;
    const int g3[3] = {x, y, z}, n3[3] = {a.nx, a.ny, a.nz}, st[3] = {1, a.nxp, pz};
    const int fk[3] = {z * a.ny + y, z * a.nx + x, y * a.nx + x};  // face cell on each axis

    constexpr int NC = Planes<MODE>::NC;
    float f[Q];
    aa_load_dir<MODE, S>(a.fin_q, c, nullptr, 0, 0, false, 0, f);
#pragma unroll
    for (int i = 1; i < 7; ++i) {
        const int ax = aa_axis(i);
        if constexpr (KIND == 0) {
            const bool up_out = g3[ax] == (aa_plus(i) ? 0 : n3[ax] - 1);  // x - c_i outside
            aa_load_dir<MODE, S>(a.fin_q + i * NC, up_out ? c : (aa_plus(i) ? c - st[ax] : c + st[ax]), g.fi[i],
                                 (int)g.fplane[ax], fk[ax], up_out && n3[ax] > 1, i, f);
        } else {
            aa_load_dir<MODE, S>(a.fin_q + i * NC, c, nullptr, 0, 0, false, i, f);
        }
    }
    FloatCell cell{f};
    update_cell<MODE, false, MU, ANA>(cell, x, y, z, __ldg(a.inv_eps + c), a, MU ? __ldg(a.inv_mu + c) : 1.0f);
    aa_store_dir<MODE, S>(a.fout_q, c, nullptr, 0, 0, false, 0, f);
#pragma unroll
    for (int i = 1; i < 7; ++i) {
        const int ax = aa_axis(i);
        const bool up_out = g3[ax] == (aa_plus(i) ? 0 : n3[ax] - 1);
        void *const *b = a.fout_q + i * NC;
        if constexpr (KIND == 0) {
            // downstream neighbour x + c_i (the cell itself along a 1-cell axis), or FO_i
            const bool down_out = g3[ax] == (aa_plus(i) ? n3[ax] - 1 : 0);
            const bool face = down_out && n3[ax] > 1;
            const int nb = down_out ? c : (aa_plus(i) ? c + st[ax] : c - st[ax]);
            aa_store_dir<MODE, S>(b, nb, g.fo[i], (int)g.fplane[ax], fk[ax], face, i, f);
            if (up_out && n3[ax] > 1)
                aa_store_dir<MODE, S>(b, c, nullptr, 0, 0, false, i, f);  // the value the in-place step pulls
        } else {
            aa_store_dir<MODE, S>(b, c, nullptr, 0, 0, false, i, f);
            if (up_out && n3[ax] > 1) aa_store_dir<MODE, S>(b, 0, g.fi[i], (int)g.fplane[ax], fk[ax], true, i, f);
        }
    }
}

// One block per row tile of BX cells (one row per block: measured at 384^3
// on GB300, several rows per block made the push step of 16-bit storage 20%
// slower and gained nothing in FP32); the first blocks also update the
// incident line.
template <int MODE, class S, int BX, bool MU, bool ANA, int KIND>
__global__ void __launch_bounds__(BX, (ANA && MODE == 2) ? 5 : 7) aa_step_kernel(const StepArgs a, const AaArgs g)
{
    const int b = blockIdx.x;
    if (a.line_on) {
        const int s = b * BX + threadIdx.x;
        if (s < a.n_line) line_work<MODE>(a, s);
    }
    const int r = b / a.nblk_x;
    aa_row<MODE, S, BX, MU, ANA, KIND>(a, g, b % a.nblk_x, r % a.ny, r / a.ny);
}

// The face cell k of axis ax (the other two coordinates, the lower one
// fastest) at coordinate u along ax: its cell index.
__device__ __forceinline__ long long aa_face_cell(int ax, int k, int u, int nx, int ny, int nxp)
{
    int x, y, z;
    if (ax == 0) {
        x = u, y = k % ny, z = k / ny;
    } else if (ax == 1) {
        x = k % nx, y = u, z = k / nx;
    } else {
        x = k % nx, y = k / nx, z = u;
    }
    return ((long long)z * ny + y) * nxp + x;
}

// FI from the canonical state: P_i(x) of the cells whose upstream neighbour
// x - c_i is outside (the first in-place step of a run would write them; any
// other change of the state has to refill them).  Storage elements are
// copied as raw bits (T: an unsigned type of the storage width).
template <class T>
__global__ void aa_fill_kernel(const T *buf, const AaArgs g, int mode, int elem, long long P, int ax, int nx, int ny,
                               int nz, int nxp)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= g.fplane[ax]) return;
    const int i = 2 * ax + 1 + blockIdx.y;
    const int n3[3] = {nx, ny, nz};
    const long long c = aa_face_cell(ax, k, aa_plus(i) ? 0 : n3[ax] - 1, nx, ny, nxp);
    T *fi = static_cast<T *>(g.fi[i]);
    const int nc = mode_NE(mode) + mode_NH(mode);
    for (int s = 0; s < nc; ++s)
        fi[aa_face_index(nc, elem, g.fplane[ax], s, k)] = buf[pop_index(mode, elem, P, slot_plane(mode, i, s), c)];
}

// Streamed -> canonical along an axis of more than one cell, for the pair of
// directions p = +axis, m = -axis and slot component s (blockIdx.y): P_p(u) is
// in slot m of u + 1 (FO_p at the last cell), P_m(u) in slot p of u - 1 (FO_m
// at the first).  One thread walks one line in increasing u, keeping the old
// slot-p value of the previous cell, so every value is read before it is
// overwritten.
template <class T>
__global__ void aa_canon_line_kernel(T *buf, const AaArgs g, int mode, int elem, long long P, int ax, int nx, int ny,
                                     int nz, int nxp)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= g.fplane[ax]) return;
    const int s = blockIdx.y;
    const int ip = 2 * ax + 1, im = ip + 1;
    const int qp = slot_plane(mode, ip, s), qm = slot_plane(mode, im, s);
    const int n = ax == 0 ? nx : (ax == 1 ? ny : nz);
    const long long plane = g.fplane[ax];
    const T *fop = static_cast<const T *>(g.fo[ip]);
    const T *fom = static_cast<const T *>(g.fo[im]);
    const int nc = mode_NE(mode) + mode_NH(mode);
    const long long fi_k = aa_face_index(nc, elem, plane, s, k);
    T carry = fom[fi_k];
    long long am = pop_index(mode, elem, P, qm, aa_face_cell(ax, k, 0, nx, ny, nxp));
    for (int u = 0; u < n; ++u) {
        const long long ap = pop_index(mode, elem, P, qp, aa_face_cell(ax, k, u, nx, ny, nxp));
        const long long am_next =
            u + 1 < n ? pop_index(mode, elem, P, qm, aa_face_cell(ax, k, u + 1, nx, ny, nxp)) : -1;
        const T old_p = buf[ap];
        const T next_m = am_next >= 0 ? buf[am_next] : fop[fi_k];
        buf[ap] = next_m;
        buf[am] = carry;
        carry = old_p;
        am = am_next;
    }
}

// Streamed -> canonical along a 1-cell axis: the two directions trade slots
// within each cell.
template <class T>
__global__ void aa_canon_swap_kernel(T *buf, int mode, int elem, long long P, int ax, int nx, int ny, int nz, int nxp)
{
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= (long long)nx * ny * nz) return;
    const int x = (int)(k % nx), y = (int)((k / nx) % ny), z = (int)(k / ((long long)nx * ny));
    const long long c = ((long long)z * ny + y) * nxp + x;
    const int ip = 2 * ax + 1, im = ip + 1;
    const int nc = mode_NE(mode) + mode_NH(mode);
    for (int s = 0; s < nc; ++s) {
        const long long ap = pop_index(mode, elem, P, slot_plane(mode, ip, s), c);
        const long long am = pop_index(mode, elem, P, slot_plane(mode, im, s), c);
        const T vp = buf[ap];
        buf[ap] = buf[am];
        buf[am] = vp;
    }
}

constexpr int kAaBX = 128;  // threads per block = cells per row tile

template <int MODE, class S, bool MU, bool ANA, int KIND>
cudaError_t launch_aa_t(StepArgs a, const AaArgs &g, cudaStream_t s)
{
    a.nblk_x = (a.nx + kAaBX - 1) / kAaBX;
    a.rows_per_block = 1;
    const long long blocks = (long long)a.nblk_x * a.ny * a.nz;
    if (blocks > INT_MAX) return cudaErrorInvalidValue;
    a.nblk_main = (int)blocks;
    if (a.line_on && (a.n_line + kAaBX - 1) / kAaBX > a.nblk_main) return cudaErrorInvalidValue;
    if (MU && a.inv_mu == nullptr) return cudaErrorInvalidValue;
    if (ANA != (a.tfsf == 2)) return cudaErrorInvalidValue;
    aa_step_kernel<MODE, S, kAaBX, MU, ANA, KIND><<<a.nblk_main, kAaBX, 0, s>>>(a, g);
    return cudaGetLastError();
}

template <int MODE, class S>
cudaError_t launch_aa_mode(int variant, int kind, const StepArgs &a, const AaArgs &g, cudaStream_t s)
{
    switch (variant * 2 + kind) {
    case 0: return launch_aa_t<MODE, S, false, false, 0>(a, g, s);
    case 1: return launch_aa_t<MODE, S, false, false, 1>(a, g, s);
    case 2: return launch_aa_t<MODE, S, true, false, 0>(a, g, s);
    case 3: return launch_aa_t<MODE, S, true, false, 1>(a, g, s);
    case 4: return launch_aa_t<MODE, S, true, true, 0>(a, g, s);
    case 5: return launch_aa_t<MODE, S, true, true, 1>(a, g, s);
    default: return cudaErrorInvalidValue;
    }
}

bool aa_faces_ok(const StepArgs &a, const AaArgs &g)
{
    const int n3[3] = {a.nx, a.ny, a.nz};
    for (int ax = 0; ax < 3; ++ax) {
        if (n3[ax] <= 1) continue;
        const long long plane = (long long)a.nx * a.ny * a.nz / n3[ax];
        if (g.fplane[ax] != plane) return false;
        for (int i = 2 * ax + 1; i <= 2 * ax + 2; ++i)
            if (!g.fi[i] || !g.fo[i]) return false;
    }
    return true;
}

}  // namespace

cudaError_t launch_aa_step(int mode, int storage, int variant, int kind, const StepArgs &a, const AaArgs &g,
                           cudaStream_t s)
{
    if (variant < 0 || variant > 2 || kind < 0 || kind > 1 || !aa_faces_ok(a, g)) return cudaErrorInvalidValue;
    switch (mode * 3 + storage) {
    case 0: return launch_aa_mode<0, float>(variant, kind, a, g, s);
    case 1: return launch_aa_mode<0, __half>(variant, kind, a, g, s);
    case 2: return launch_aa_mode<0, __nv_bfloat16>(variant, kind, a, g, s);
    case 3: return launch_aa_mode<1, float>(variant, kind, a, g, s);
    case 4: return launch_aa_mode<1, __half>(variant, kind, a, g, s);
    case 5: return launch_aa_mode<1, __nv_bfloat16>(variant, kind, a, g, s);
    case 6: return launch_aa_mode<2, float>(variant, kind, a, g, s);
    case 7: return launch_aa_mode<2, __half>(variant, kind, a, g, s);
    case 8: return launch_aa_mode<2, __nv_bfloat16>(variant, kind, a, g, s);
    default: return cudaErrorInvalidValue;
    }
}

namespace {
template <class T>
cudaError_t aa_fill_t(int mode, int elem, const void *buf, long long P, int nx, int ny, int nz, int nxp,
                      const AaArgs &g, cudaStream_t s)
{
    const int n3[3] = {nx, ny, nz};
    for (int ax = 0; ax < 3; ++ax) {
        if (n3[ax] <= 1) continue;
        const dim3 grid((unsigned)((g.fplane[ax] + 255) / 256), 2);
        aa_fill_kernel<T><<<grid, 256, 0, s>>>(static_cast<const T *>(buf), g, mode, elem, P, ax, nx, ny, nz, nxp);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

template <class T>
cudaError_t aa_canonical_t(int mode, int elem, void *buf, long long P, int nx, int ny, int nz, int nxp,
                           const AaArgs &g, cudaStream_t s)
{
    const int n3[3] = {nx, ny, nz};
    const int nc = mode_NE(mode) + mode_NH(mode);
    for (int ax = 0; ax < 3; ++ax) {
        if (n3[ax] <= 1) {
            const long long cells = (long long)nx * ny * nz;
            aa_canon_swap_kernel<T><<<(unsigned)((cells + 255) / 256), 256, 0, s>>>(static_cast<T *>(buf), mode, elem,
                                                                                     P, ax, nx, ny, nz, nxp);
        } else {
            const dim3 grid((unsigned)((g.fplane[ax] + 127) / 128), nc);
            aa_canon_line_kernel<T><<<grid, 128, 0, s>>>(static_cast<T *>(buf), g, mode, elem, P, ax, nx, ny, nz,
                                                        nxp);
        }
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}
}  // namespace

cudaError_t launch_aa_fill(int mode, int storage, const void *buf, long long P, int nx, int ny, int nz, int nxp,
                           const AaArgs &g, cudaStream_t s)
{
    StepArgs dims;
    dims.nx = nx, dims.ny = ny, dims.nz = nz;
    if (!aa_faces_ok(dims, g)) return cudaErrorInvalidValue;
    return storage == 0 ? aa_fill_t<unsigned>(mode, 4, buf, P, nx, ny, nz, nxp, g, s)
                        : aa_fill_t<unsigned short>(mode, 2, buf, P, nx, ny, nz, nxp, g, s);
}

cudaError_t launch_aa_canonical(int mode, int storage, void *buf, long long P, int nx, int ny, int nz, int nxp,
                                const AaArgs &g, cudaStream_t s)
{
    StepArgs dims;
    dims.nx = nx, dims.ny = ny, dims.nz = nz;
    if (!aa_faces_ok(dims, g)) return cudaErrorInvalidValue;
    return storage == 0 ? aa_canonical_t<unsigned>(mode, 4, buf, P, nx, ny, nz, nxp, g, s)
                        : aa_canonical_t<unsigned short>(mode, 2, buf, P, nx, ny, nz, nxp, g, s);
}

}  // namespace lbem
