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
#include <algorithm>
#include <climits>
#include <mutex>

#include "step_cell.cuh"

namespace lbem {
namespace {

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
    sa.line_n1 = P.line[(t + 1) % kLineBufs];
    sa.line_out = P.line[(t + 2) % kLineBufs];
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



// Sums cnt staged steps of face fields into the FP64 DFT accumulators in step
// order, with the same fma as the direct path.  A thread takes one face cell
// per pass of the grid-stride loop and the components k = blockIdx.y,
// blockIdx.y + gridDim.y, ...; reads are coalesced along the cells and a
// component's staged values are all loaded before its FP64 chain.  Slot s
// holds the faces in mask[s].  A small grid of it (one block per SM, every
// component) runs beside the two-step kernel that fills the other bank, one
// block beside each two-step block: that needs its warps to fit the
// registers the two-step block leaves on each SM sub-partition (1024 beside
// the 19 warps of 96 registers of the 16-bit kernel, hence at most 32
// registers a thread) and an SM shared-memory configuration that still holds
// a two-step block (the maximum carveout: a flush block that lands first on
// an idle SM would otherwise configure it for L1 and keep the next two-step
// block off that SM while it runs).
constexpr int kFlushThreads = 128;
__global__ void __launch_bounds__(kFlushThreads, 16) dft_flush_x_kernel(const DftFlushArgs a)
{
    // 32-bit offsets: the launcher checks that kXBank staged steps and the
    // accumulators of every face stay below 2^31 elements
    const int n = (int)a.n;
    const int slot = a.nc * n;  // floats of one staged step
    for (int j = blockIdx.x * kFlushThreads + threadIdx.x; j < n; j += gridDim.x * kFlushThreads) {
        int f = 0;
        while (f + 1 < a.nfaces && j >= a.start[f + 1]) ++f;
        unsigned on = 0;  // the slots that staged face f
#pragma unroll
        for (int s = 0; s < kXBank; ++s)
            if (s < a.cnt) on |= ((a.mask[s] >> f) & 1u) << s;
        if (!on) continue;
        const float *src = a.stage + j;
        double *base = a.dft + a.face_off[f] + (j - (int)a.start[f]);
        const int plane = (int)a.plane[f];
        for (int k = blockIdx.y; k < a.nc; k += gridDim.y) {
            float v[kXBank];
#pragma unroll
            for (int s = 0; s < kXBank; ++s)
                v[s] = ((on >> s) & 1u) ? src[s * slot + k * n] : 0.f;
            double re = base[(2 * k + 0) * plane], im = base[(2 * k + 1) * plane];
#pragma unroll
            for (int s = 0; s < kXBank; ++s) {
                if (!((on >> s) & 1u)) continue;
                re = fma((double)v[s], a.sc[s], re);
                im = fma((double)v[s], -a.ss[s], im);
            }
            base[(2 * k + 0) * plane] = re;
            base[(2 * k + 1) * plane] = im;
        }
    }
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

}  // namespace

long long l2_bytes()
{
    static std::mutex mu;
    static long long cache[kMaxDevices];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return 0;
    std::lock_guard<std::mutex> lock(mu);
    if (cache[dev] == 0) {
        int n = 0;
        if (cudaDeviceGetAttribute(&n, cudaDevAttrL2CacheSize, dev) != cudaSuccess) return 0;
        cache[dev] = n;
    }
    return cache[dev];
}

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

cudaError_t launch_dft_flush_x(const DftFlushArgs &a, cudaStream_t s, int blocks)
{
    if (a.cnt < 1 || a.cnt > kXBank || a.n <= 0 || blocks < 0) return cudaErrorInvalidValue;
    if ((long long)kXBank * a.nc * a.n > INT_MAX) return cudaErrorInvalidValue;
    for (int f = 0; f < a.nfaces; ++f)
        if (a.face_off[f] + 2LL * a.nc * a.plane[f] > INT_MAX) return cudaErrorInvalidValue;
    const long long need = (a.n + kFlushThreads - 1) / kFlushThreads;
    const dim3 grid(blocks > 0 ? (unsigned)std::min<long long>(blocks, need) : (unsigned)need,
                    blocks > 0 ? 1u : (unsigned)a.nc);
    {
        static std::mutex mu;
        static bool carved[kMaxDevices];
        int dev = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e != cudaSuccess) return e;
        if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
        std::lock_guard<std::mutex> lock(mu);
        if (!carved[dev]) {
            e = cudaFuncSetAttribute(dft_flush_x_kernel, cudaFuncAttributePreferredSharedMemoryCarveout,
                                     cudaSharedmemCarveoutMaxShared);
            if (e != cudaSuccess) return e;
            carved[dev] = true;
        }
    }
    dft_flush_x_kernel<<<grid, kFlushThreads, 0, s>>>(a);
    return cudaGetLastError();
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
