// Two lattice updates per pass over HBM (temporal blocking) for the fused
// D3Q7 step of arXiv 2510.11042, Sec. 2.1 (Eq. 1 applied twice, the boundary
// of Eq. 4 at every pull): the 3D pass over xy tiles marching in z and the 2D
// pass over x strips marching in y, both with level n staged in shared memory
// by the tensor-memory accelerator.  Every update is the single-step kernel's
// update_cell (step_cell.cuh), so both give the same bits.
#include <cuda.h>

#include <algorithm>
#include <cstring>
#include <mutex>
#include <type_traits>

#include "step_cell.cuh"

namespace lbem {
namespace {

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
    static constexpr int NBUF = 2;
    static constexpr int SMEM = NBUF * BUNDLE + 3 * SLOT;
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
    static constexpr int NBUF = 2;
    static constexpr int SMEM = NBUF * BUNDLE + 3 * SLOT;
    static constexpr int MIN_BLOCKS = 1;
    // launched in clusters of two x-adjacent tiles, with the boxes' L2 fetch
    // granularity left at the default (measured at 384^3: 1.93 -> 1.71 ms per
    // update with the evict-first stores); 16-bit storage measured faster
    // without clusters and with 256-byte L2 promotion
    static constexpr int CLUSTER_X = 2;
};
// The bundle of a pass variant V (0: plain update, 1: per-cell 1/mu_r map):
// V > 0 adds a box of 1/mu_r of the same shape beside the 1/eps_r box.
template <class L, int V> struct WithMu : L {
    static constexpr bool HAS_MU = V > 0;
    static constexpr int MU_OFF = t2::pad128(L::EPS_OFF + L::EPS_BYTES);
    static constexpr int BUNDLE = HAS_MU ? t2::pad128(MU_OFF + L::EPS_BYTES) : L::BUNDLE;
    static constexpr unsigned TX_BYTES = L::TX_BYTES + (HAS_MU ? L::EPS_BYTES : 0);
    static constexpr int SMEM = L::NBUF * BUNDLE + 3 * L::SLOT;
};
static_assert(WithMu<T2L<float>, 1>::SMEM <= 232448 - 1024, "two-step FP32 shared memory");
static_assert(WithMu<T2L<__half>, 1>::SMEM <= 232448 - 1024, "two-step 16-bit shared memory");

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
    CUtensorMap map_mu;   // 1/mu_r (the variant with a mu_r map)
    StepArgs s1, s2;      // the two steps: s1 reads level n (fin_q), s2 writes level n+2 (fout_q)
    int zc;               // planes per z chunk (blockIdx.z)
    // 2D: the incident line's work of the next pass's two steps (line(n+4)
    // from line(n+3), then line(n+5)), done by the first block before its
    // strips; the pass itself reads line(n+1) and line(n+2) only
    int ahead_on;
    StepArgs ahead1, ahead2;
};

// The first block of a 2D pass advances the incident line for the next pass
// (line2_kernel's work, two steps in order), so that pass needs no launch of
// its own for it (4096^2 EZ per update: FP32 0.2372 -> 0.2268 ms, FP16
// 0.1666 -> 0.1631, BF16 0.1745 -> 0.1682).
template <int MODE>
__device__ __forceinline__ void t2_line_ahead(const Step2Args &P)
{
    if (!P.ahead_on || blockIdx.x != 0 || blockIdx.y != 0 || blockIdx.z != 0) return;
    for (int s = threadIdx.x; s < P.ahead1.n_line; s += blockDim.x) line_work<MODE>(P.ahead1, s);
    __syncthreads();
    for (int s = threadIdx.x; s < P.ahead2.n_line; s += blockDim.x) line_work<MODE>(P.ahead2, s);
    __syncthreads();
}

// Copy the level-n bundle of plane p into the buffer at dst; the copies
// complete the mbarrier bar.  Every x coordinate is x0 - X0 with x0 a
// multiple of 32, so each box starts on a 16-byte boundary.
template <class S, int V>
__device__ __forceinline__ void t2_issue(const Step2Args &P, uint32_t dst, uint32_t bar, int x0, int y0, int p, int nz)
{
    using L = WithMu<T2L<S>, V>;
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
    if constexpr (L::HAS_MU) tma_load_3d(dst + L::MU_OFF, &P.map_mu, x0 - t2::EPS_X0, y0 - 1, p, bar);
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
template <class S, int V>
__device__ __forceinline__ void t2_level2(const StepArgs &s2, const unsigned char *slot, int t, int x, int y, int z,
                                          const DirVal<S> &d0, const DirVal<S> &d5, const DirVal<S> &d6, float ie,
                                          float im)
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
    update_cell<2, false, (V > 0), false, true>(cell, x, y, z, ie, s2, im, true);
    store_cell_evict_first<S>(s2, (z * ny + y) * s2.nxp + x, f);
}

template <class S, int V>
__device__ __forceinline__ void step2_body(const Step2Args &P)
{
    using L = WithMu<T2L<S>, V>;
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
        t2_issue<S, V>(P, buf0, bar0, x0, y0, pa, nz);
        t2_issue<S, V>(P, buf0 + L::BUNDLE, bar0 + 8, x0, y0, pa + 1, nz);
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
    float ie_prev = 1.f, im_prev = 1.f;
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
        float ie_cur = 1.f, im_cur = 1.f;
        if (live && !failed && !bad) {
            float f[Planes<2>::Q];
            bundle_cell<S>(buf, col, row, x, y, nx, ny, f);
            const int ei = row * EPS_W + (x - x0 + EPS_X0);
            const float ie = reinterpret_cast<const float *>(buf + L::EPS_OFF)[ei];
            float im = 1.f;
            if constexpr (L::HAS_MU) im = reinterpret_cast<const float *>(buf + L::MU_OFF)[ei];
            FloatCell cell{f};
            update_cell<2, false, (V > 0), false, true>(cell, x, y, p, ie, s1, im, tile && p >= z0 && p < z1);
            if (tile) {
#pragma unroll
                for (int d = 1; d <= 4; ++d) slot_put<S>(slot, false, d, t, to_dir<S>(f, d));
                d0_cur = to_dir<S>(f, 0);
                d5_cur = to_dir<S>(f, 5);
                d6_cur = to_dir<S>(f, 6);
                ie_cur = ie;
                im_cur = im;
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
            t2_issue<S, V>(P, buf0 + (j & 1) * L::BUNDLE, bar0 + 8 * (j & 1), x0, y0, p + 2, nz);
        }
        // level n+2 of plane p - 1 (p - 1 < z1 holds, since p <= pb <= z1);
        // at p - 1 == 0 the +z pull clamps to the plane itself
        if (!failed && tile && live && p - 1 >= z0)
            t2_level2<S, V>(s2, slots + ((p - 1) % 3) * L::SLOT, t, x, y, p - 1, d0_prev,
                            p - 1 == 0 ? d5_prev : d5_pp, d6_cur, ie_prev, im_prev);
        d5_pp = d5_prev;
        d5_prev = d5_cur;
        d0_prev = d0_cur;
        ie_prev = ie_cur;
        im_prev = im_cur;
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
        t2_level2<S, V>(s2, slots + ((nz - 1) % 3) * L::SLOT, t, x, y, nz - 1, d0_prev, d5_pp, d6_cur, ie_prev,
                        im_prev);
}

// One block per SM (its shared memory): FP32 352 threads, 16-bit 608.
template <class S, int V>
__global__ void __launch_bounds__(T2L<S>::THREADS, T2L<S>::MIN_BLOCKS) step2_kernel(const __grid_constant__ Step2Args P)
{
    step2_body<S, V>(P);
}

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
    static constexpr int NBUF = t2d::NB;
    static constexpr int SMEM = NBUF * BUNDLE + 3 * SLOT;
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
template <class S, int V>
__device__ __forceinline__ void t2d_issue(const Step2Args &P, uint32_t dst, uint32_t bar, int x0, int r, int ny)
{
    using L = WithMu<T2D<S>, V>;
    const int rm = r > 0 ? r - 1 : 0, rp = r < ny - 1 ? r + 1 : ny - 1;
    mbar_expect_tx(bar, L::TX_BYTES);
#pragma unroll
    for (int d = 0; d < 7; ++d) {
        const int row = d == 3 ? rm : (d == 4 ? rp : r);
        tma_load_3d(dst + d * L::DIR_BYTES, &P.map_a, x0 - L::X0, row, d, bar);
        tma_load_3d(dst + d * L::DIR_BYTES + L::SINGLE_OFF, &P.map_b, x0 - L::X0, row, d, bar);
    }
    tma_load_2d(dst + L::EPS_OFF, &P.map_eps, x0 - L::X0, r, bar);
    if constexpr (L::HAS_MU) tma_load_2d(dst + L::MU_OFF, &P.map_mu, x0 - L::X0, r, bar);
}

// Level n+2 of strip cell t at (x, y) from level n+1.
template <int MODE, class S, int V>
__device__ __forceinline__ void t2d_level2(const StepArgs &s2, const unsigned char *slot, int t, int x, int y,
                                           const DirVal2<S> &d0, const DirVal2<S> &d3, const DirVal2<S> &d4,
                                           const DirVal2<S> &d5, const DirVal2<S> &d6, float ie, float im)
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
    update_cell<MODE, false, (V > 0), false, true>(cell, x, y, 0, ie, s2, im, true);
    store_cell<MODE, S>(s2, y * s2.nxp + x, f);
}

template <int MODE, class S, int V>
__device__ __forceinline__ void step2d_body(const Step2Args &P)
{
    using L = WithMu<T2D<S>, V>;
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
    t2_line_ahead<MODE>(P);

    if (t == t2d::ISSUER) {
        for (int b = 0; b < t2d::NB; ++b) mbar_init(bar0 + 8 * b, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    __syncthreads();
    if (t == t2d::ISSUER)
        for (int j = 0; j < t2d::NB && j < nl1; ++j)
            t2d_issue<S, V>(P, buf0 + j * L::BUNDLE, bar0 + 8 * j, x0, pa + j, ny);

    // this thread's cell: a strip cell, the left or right halo cell, or none
    const bool strip = t < TXS;
    const int x = strip ? x0 + t : (t == t2d::HALO ? x0 - 1 : (t == t2d::HALO + 1 ? x0 + TXS : -1));
    const bool live = x >= 0 && x < nx;
    const int col = x - x0 + L::X0;

    DirVal2<S> d0_prev{}, d3_prev{}, d3_pp{}, d5_prev{}, d6_prev{}, d4_cur{};
    float ie_prev = 1.f, im_prev = 1.f;
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
        float ie_cur = 1.f, im_cur = 1.f;
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
            float im = 1.f;
            if constexpr (L::HAS_MU) im = reinterpret_cast<const float *>(buf + L::MU_OFF)[col];
            FloatCell cell{f};
            update_cell<MODE, false, (V > 0), false, true>(cell, x, p, 0, ie, s1, im, strip && p >= y0 && p < y1);
            if (strip) {
                slot2_put<S>(slot, t, to_dir2<MODE, S>(f, 1));
                slot2_put<S>(slot, TXS + t, to_dir2<MODE, S>(f, 2));
                d0_cur = to_dir2<MODE, S>(f, 0);
                d3_cur = to_dir2<MODE, S>(f, 3);
                d4_cur = to_dir2<MODE, S>(f, 4);
                d5_cur = to_dir2<MODE, S>(f, 5);
                d6_cur = to_dir2<MODE, S>(f, 6);
                ie_cur = ie;
                im_cur = im;
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
            t2d_issue<S, V>(P, buf0 + (j % t2d::NB) * L::BUNDLE, bar0 + 8 * (j % t2d::NB), x0, p + t2d::NB, ny);
        }
        // level n+2 of row p - 1; at p - 1 == 0 the +y pull clamps to the row itself
        if (!failed && strip && live && p - 1 >= y0)
            t2d_level2<MODE, S, V>(s2, slots + ((p - 1) % 3) * L::SLOT, t, x, p - 1, d0_prev,
                                   p - 1 == 0 ? d3_prev : d3_pp, d4_cur, d5_prev, d6_prev, ie_prev, im_prev);
        d3_pp = d3_prev;
        d3_prev = d3_cur;
        d0_prev = d0_cur;
        d5_prev = d5_cur;
        d6_prev = d6_cur;
        ie_prev = ie_cur;
        im_prev = im_cur;
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
        t2d_level2<MODE, S, V>(s2, slots + ((ny - 1) % 3) * L::SLOT, t, x, ny - 1, d0_prev, d3_pp, d4_cur, d5_prev,
                               d6_prev, ie_prev, im_prev);
}

template <int MODE, class S, int V>
__global__ void __launch_bounds__(t2d::THREADS, T2D<S>::MIN_BLOCKS) step2d_kernel(const __grid_constant__ Step2Args P)
{
    step2d_body<MODE, S, V>(P);
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
// blocks per SM, per (mode, storage, variant) (set up once, under a lock).
std::mutex g_step2_mu;
int g_step2_bps[kMaxDevices][3][3][3];

// The 1/mu_r map of a variant with one (V > 0): the same box as 1/eps_r.
bool encode_mu(Step2Args &P, const StepArgs &s1, const cuuint64_t *dims, const cuuint64_t *str,
               const cuuint32_t *box, int rank)
{
    return s1.inv_mu && encode_map(&P.map_mu, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, rank, s1.inv_mu, dims, str, box);
}

template <class Kernel>
cudaError_t setup_kernel(Kernel k, int smem, int threads, int &bps)
{
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    int n = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, threads, smem);
    if (e != cudaSuccess) return e;
    if (n < 1) return cudaErrorInvalidConfiguration;
    bps = n;
    return cudaSuccess;
}

template <int MODE, class S, int V>
cudaError_t step2_setup(int &blocks_per_sm)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_step2_mu);
    int &bps = g_step2_bps[dev][MODE][storage_slot<S>()][V];
    if (bps == 0) {
        if constexpr (MODE == 2)
            e = setup_kernel(step2_kernel<S, V>, WithMu<T2L<S>, V>::SMEM, T2L<S>::THREADS, bps);
        else
            e = setup_kernel(step2d_kernel<MODE, S, V>, WithMu<T2D<S>, V>::SMEM, t2d::THREADS, bps);
        if (e != cudaSuccess) return e;
    }
    blocks_per_sm = bps;
    return cudaSuccess;
}

// Whether 3D two-step passes pay on this grid: the tiles times z chunks of at
// least 16 planes fill one wave of resident blocks.  The grid must also hold
// a whole box in x and y.
template <class S, int V>
bool step2_worthwhile_t(int nx, int ny, int nz)
{
    if (nx < 64 || ny < T2L<S>::ROWS || nz < 2) return false;
    int bps = 0;
    if (step2_setup<2, S, V>(bps) != cudaSuccess) return false;
    using L = T2L<S>;
    const long long tiles = (long long)((nx + L::TX - 1) / L::TX) * ((ny + L::TY - 1) / L::TY);
    return tiles * std::max(1, nz / 16) >= (long long)std::max(1, sm_count()) * bps;
}

template <class S, int V>
cudaError_t launch_step2_t(const StepArgs &s1, const StepArgs &s2, cudaStream_t s, const StepArgs *ahead,
                           bool line_ready)
{
    using L = WithMu<T2L<S>, V>;
    // the 3D pass keeps the one-block line launch: with the line work in its
    // first block, the 16-bit pass took 1.06-1.07 ms per update at 384^3
    // instead of 0.956 (same registers, no spills) and FP32 gained 0.1 %
    if (ahead || line_ready) return cudaErrorInvalidValue;
    if (s1.nx < 64 || s1.ny < L::ROWS || s1.nz < 2 || s1.nxp % 32 || s1.P % 32) return cudaErrorInvalidValue;
    int bps = 0;
    cudaError_t e = step2_setup<2, S, V>(bps);
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
        if (L::HAS_MU) ok = ok && encode_mu(P, s1, dims, str, box, 3);
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
        e = cudaLaunchKernelEx(&cfg, step2_kernel<S, V>, P);
        if (e != cudaSuccess) return e;
    } else {
        step2_kernel<S, V><<<grid, L::THREADS, L::SMEM, s>>>(P);
    }
    return cudaGetLastError();
}

// ---- host side of the 2D two-step pass

// Whether 2D two-step passes pay: the population buffers of the grids
// stepping together exceed L2 by a fifth (below that a single step's traffic
// stays in L2; measured on EZ cylinders per update, single step against
// two-step pass: 768^2 FP32 (99 MB) 0.0144 / 0.0173 ms, 1024^2 FP32 (176 MB)
// 0.0307 / 0.0231, 1024^2 FP16 (88 MB) 0.0164 / 0.0205, 2048^2 FP16 (352 MB)
// 0.0647 / 0.0531), and the strips times chunks of 16 rows fill half a wave
// of resident blocks; boxes must fit the row.
template <int MODE, class S, int V>
bool step2d_worthwhile_t(int nx, int ny, int share)
{
    if (nx < 256 || ny < 16) return false;
    const long long nxp = (nx + 31) / 32 * 32;
    const long long pop_bytes = 2LL * Planes<MODE>::Q * nxp * ny * (long long)sizeof(S);
    if (5 * pop_bytes * share < 6 * l2_bytes()) return false;
    int bps = 0;
    if (step2_setup<MODE, S, V>(bps) != cudaSuccess) return false;
    const long long strips = (nx + t2d::TXS - 1) / t2d::TXS;
    return 2 * strips * std::max(1, ny / 16) * share >= (long long)std::max(1, sm_count()) * bps;
}

template <int MODE, class S, int V>
cudaError_t launch_step2d_t(const StepArgs &s1, const StepArgs &s2, cudaStream_t s, int share, const StepArgs *ahead,
                            bool line_ready)
{
    using L = WithMu<T2D<S>, V>;
    if (s1.nz != 1 || s1.nx < 256 || s1.ny < 16 || s1.nxp % 32 || s1.P % 32) return cudaErrorInvalidValue;
    int bps = 0;
    cudaError_t e = step2_setup<MODE, S, V>(bps);
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
        if (L::HAS_MU) ok = ok && encode_mu(P, s1, de, se, be, 2);
    }
    if (!ok) return cudaErrorInvalidValue;
    if (s1.line_on && !line_ready) {
        line2_kernel<MODE><<<1, 512, 0, s>>>(P.s1, P.s2);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    if (ahead) {
        P.ahead_on = 1;
        P.ahead1 = ahead[0];
        P.ahead2 = ahead[1];
    }
    // row chunks as the 3D pass's z chunks: about 40 rows, more and shorter
    // (at least 8 rows) where that would not fill two waves (together with the
    // grids stepping beside this one)
    const long long strips = (s1.nx + t2d::TXS - 1) / t2d::TXS;
    const long long cap = (long long)std::max(1, sm_count()) * bps;
    int nyc = std::max(1, (s1.ny + 20) / 40);
    while (strips * nyc * share < 2 * cap && (s1.ny + nyc) / (nyc + 1) >= 8) ++nyc;
    P.zc = (s1.ny + nyc - 1) / nyc;
    const dim3 grid((unsigned)strips, (s1.ny + P.zc - 1) / P.zc, 1);
    step2d_kernel<MODE, S, V><<<grid, t2d::THREADS, L::SMEM, s>>>(P);
    return cudaGetLastError();
}

template <class S, int V>
cudaError_t launch_mode(int mode, const StepArgs &s1, const StepArgs &s2, cudaStream_t s, int share,
                        const StepArgs *ahead, bool line_ready)
{
    switch (mode) {
    case 0: return launch_step2d_t<0, S, V>(s1, s2, s, share, ahead, line_ready);
    case 1: return launch_step2d_t<1, S, V>(s1, s2, s, share, ahead, line_ready);
    case 2: return launch_step2_t<S, V>(s1, s2, s, ahead, line_ready);
    default: return cudaErrorInvalidValue;
    }
}

// The closed-form source (variant 2) takes single steps: it is bound by its
// eight wave evaluations per cell, not by memory (384^3 sphere at 30 degrees
// per update: FP32 2.86 ms in two-step passes against 2.82 ms in single
// steps; FP16 3.02 against 1.95 ms, the two-step kernel spilling).
template <class S>
cudaError_t launch_variant(int mode, int variant, const StepArgs &s1, const StepArgs &s2, cudaStream_t s,
                           int share, const StepArgs *ahead, bool line_ready)
{
    switch (variant) {
    case 0: return launch_mode<S, 0>(mode, s1, s2, s, share, ahead, line_ready);
    case 1: return launch_mode<S, 1>(mode, s1, s2, s, share, ahead, line_ready);
    default: return cudaErrorInvalidValue;
    }
}

template <class S, int V>
bool worthwhile_mode(int mode, int nx, int ny, int nz, int share)
{
    switch (mode) {
    case 0: return step2d_worthwhile_t<0, S, V>(nx, ny, share);
    case 1: return step2d_worthwhile_t<1, S, V>(nx, ny, share);
    case 2: return step2_worthwhile_t<S, V>(nx, ny, nz);
    default: return false;
    }
}

template <class S>
bool worthwhile_variant(int mode, int variant, int nx, int ny, int nz, int share)
{
    switch (variant) {
    case 0: return worthwhile_mode<S, 0>(mode, nx, ny, nz, share);
    case 1: return worthwhile_mode<S, 1>(mode, nx, ny, nz, share);
    default: return false;
    }
}

}  // namespace

cudaError_t launch_step2(int mode, int storage, int variant, const StepArgs &s1, const StepArgs &s2,
                         cudaStream_t s, int share, const StepArgs *ahead, bool line_ready)
{
    share = std::max(1, share);
    if ((ahead || line_ready) && !s1.line_on) return cudaErrorInvalidValue;
    switch (storage) {
    case 0: return launch_variant<float>(mode, variant, s1, s2, s, share, ahead, line_ready);
    case 1: return launch_variant<__half>(mode, variant, s1, s2, s, share, ahead, line_ready);
    case 2: return launch_variant<__nv_bfloat16>(mode, variant, s1, s2, s, share, ahead, line_ready);
    default: return cudaErrorInvalidValue;
    }
}

bool step2_worthwhile(int mode, int storage, int variant, int nx, int ny, int nz, int share)
{
    share = std::max(1, share);
    switch (storage) {
    case 0: return worthwhile_variant<float>(mode, variant, nx, ny, nz, share);
    case 1: return worthwhile_variant<__half>(mode, variant, nx, ny, nz, share);
    case 2: return worthwhile_variant<__nv_bfloat16>(mode, variant, nx, ny, nz, share);
    default: return false;
    }
}

}  // namespace lbem
