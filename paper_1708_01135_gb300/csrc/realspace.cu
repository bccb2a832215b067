// Real-space pair sum (hot-path step a4): Section 3.1.1, Eq. 4 and Listing 1.
//
//   phi_i = sum_{j : 0 < |r_ij| < r_c} q_j erfc(beta r_ij) / r_ij
//   F_i   = q_i sum_j q_j (r_ij / r_ij^2) [erfc(beta r_ij) / r_ij
//                                          + 2 beta / sqrt(pi) exp(-beta^2 r_ij^2)]
//   E_real = 1/2 sum_i q_i phi_i            (r_ij = r_i - r_j, minimum image)
//
// GPU design (templated on FP64 and FP32 arithmetic):
//   * One warp owns a tile of up to 16 (or 32) consecutive sorted particles of one row of
//     cells (fixed c_y, c_z).  With 16, lane = (target i, partner group g): every target has
//     2 lanes that take every other partner, and the 2 partial sums of a target are combined
//     with a shuffle at the end; with 32 (cells of 16 particles or more) every lane owns one
//     target.  Either way every target's force is written by one lane and no two threads ever
//     write the same particle (the paper's rule that a loop writes only its own particle,
//     Section 3.2.3, with no atomics).  The tile size per plan follows the cell occupancy:
//     narrow tiles keep the candidate set close to the cutoff sphere where cells are sparse,
//     wide ones amortise the candidate traffic where they are dense.
//   * The candidate partners j of a tile are the cells of the neighbour rows (c_y + dy,
//     c_z + dz), |dy|, |dz| <= w, in the x range of the tile widened by the reach left for
//     that row.  A run of cells along x is a contiguous range of the sorted array, so it is
//     copied to shared memory with one bulk TMA copy (cp.async.bulk, completion on an
//     mbarrier), double-buffered per warp; all lanes then read each j as a broadcast.
//   * Positions are stored relative to the corner of their own cell; the offset between a
//     target and a partner cell is an exact small multiple of the cell side.  This keeps
//     FP32 differences accurate to ~1e-7 of the cell size instead of ~1e-7 of L, and makes
//     the periodic image implicit (the neighbour cell index wraps, the offset does not).
//   * Energies: one FP64 partial per tile, summed in tile order by the finalize step.
#include <cuda_runtime.h>
#include <stdint.h>

#include "ewald_internal.cuh"

namespace ew {
namespace {

constexpr int kWarps = 4;      // warps (tiles) per block
constexpr int kCap = 128;      // particles per staging buffer (cell mode)
constexpr int kCapAll = 256;   // particles per staging buffer (all-pairs mode)
// Targets per warp tile in cell mode: 16 (two partner lanes per target) for sparse cells,
// 32 (one lane per target) where cells hold 16 particles or more; chosen per plan.
constexpr int kTileSparse = 16, kTileDense = 32;

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
}

__device__ __forceinline__ void fence_mbar_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void tma_bulk_g2s(void *dst, const void *src, uint32_t bytes,
                                             uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
            "r"(smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ uint32_t mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok;
}

__device__ __forceinline__ uint64_t globaltimer()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}

// Whole-warp bounded wait on an mbarrier phase: true when it completed, false after ~1 s.
__device__ __forceinline__ bool warp_wait(uint64_t *bar, uint32_t parity)
{
    const uint64_t t0 = globaltimer();
    while (true) {
        uint32_t ok = mbar_try_wait(bar, parity);
        if (__all_sync(0xffffffffu, ok)) return true;
        if (__any_sync(0xffffffffu, globaltimer() - t0 > 1000000000ull)) return false;
    }
}

// The failure path of the bounded waits: one warp waits on an mbarrier phase that nothing
// completes (no copy is issued and nobody arrives), gives up after ~1 s exactly as a pair
// kernel whose staged copy never lands, and sets the timeout bit of the status word.
__global__ void k_wait_probe(int *__restrict__ status)
{
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
    }
    __syncwarp();
    if (!warp_wait(&bar, 0u) && threadIdx.x == 0) atomicOr(status, kStTimeout);
}

template <class T> struct Vec4;
template <> struct Vec4<float> { using type = float4; };
template <> struct Vec4<double> { using type = double4_32a; };

__device__ __forceinline__ double erfc_t(double x) { return erfc(x); }
__device__ __forceinline__ float exp_t(float x) { return __expf(x); }
__device__ __forceinline__ double exp_t(double x) { return exp(x); }
__device__ __forceinline__ float rsqrt_t(float x) { return rsqrtf(x); }
__device__ __forceinline__ double rsqrt_t(double x) { return 1.0 / sqrt(x); }

// Per-target sums of one warp lane: force / q_i and potential; with kVir the six
// independent entries (xx, yy, zz, xy, xz, yz) of sum_j s_ij d_a d_b, s_ij d_vec being the
// force / q_i that partner j exerts, so that the target's share of the virial tensor is
// 1/2 q_i times that sum; with kLJ the Lennard-Jones force and pair-energy sums (and with
// both, the Lennard-Jones virial sums, whose share is 1/2 of the sum).
// (The optional sums are empty base classes when off, so they take no registers or shared
// memory in the variants that do not use them.)
template <class T> struct AccBase { T fx, fy, fz, phi; };
template <class T, bool on> struct AccVir {};
template <class T> struct AccVir<T, true> { T w[6]; };
template <class T, bool on> struct AccLJ {};
template <class T> struct AccLJ<T, true> { T lj_f[4]; };
template <class T, bool on> struct AccLJVir {};
template <class T> struct AccLJVir<T, true> { T lj_w[6]; };
template <class T, bool kVir, bool kLJ>
struct PairAcc : AccBase<T>, AccVir<T, kVir>, AccLJ<T, kLJ>, AccLJVir<T, kVir && kLJ> {
    static constexpr bool vir = kVir, lj = kLJ;
};

template <class A>
__device__ __forceinline__ void acc_shfl_add(A &a, int o)
{
    a.fx += __shfl_xor_sync(0xffffffffu, a.fx, o);
    a.fy += __shfl_xor_sync(0xffffffffu, a.fy, o);
    a.fz += __shfl_xor_sync(0xffffffffu, a.fz, o);
    a.phi += __shfl_xor_sync(0xffffffffu, a.phi, o);
    if constexpr (A::vir) {
#pragma unroll
        for (int c = 0; c < 6; ++c) a.w[c] += __shfl_xor_sync(0xffffffffu, a.w[c], o);
    }
    if constexpr (A::lj) {
#pragma unroll
        for (int c = 0; c < 4; ++c) a.lj_f[c] += __shfl_xor_sync(0xffffffffu, a.lj_f[c], o);
    }
    if constexpr (A::vir && A::lj) {
#pragma unroll
        for (int c = 0; c < 6; ++c) a.lj_w[c] += __shfl_xor_sync(0xffffffffu, a.lj_w[c], o);
    }
}

template <class A>
__device__ __forceinline__ void acc_add(A &a, const A &o)
{
    a.fx += o.fx; a.fy += o.fy; a.fz += o.fz; a.phi += o.phi;
    if constexpr (A::vir) {
#pragma unroll
        for (int c = 0; c < 6; ++c) a.w[c] += o.w[c];
    }
    if constexpr (A::lj) {
#pragma unroll
        for (int c = 0; c < 4; ++c) a.lj_f[c] += o.lj_f[c];
    }
    if constexpr (A::vir && A::lj) {
#pragma unroll
        for (int c = 0; c < 6; ++c) a.lj_w[c] += o.lj_w[c];
    }
}

// Fixed shuffle tree over the 32 lanes; lane 0 holds the warp's sum.
__device__ __forceinline__ double warp_sum(double v)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// The tile's shares of the virial sums: vir_tile[c * vcap + tile] = sum over the tile's
// targets of 1/2 q_i w_c (c < 6), and with Lennard-Jones pairs 1/2 lj_w_c (rows 6..11); the
// Lennard-Jones energy 1/2 sum of the pair energies into e_lj[tile].
template <class A>
__device__ __forceinline__ void acc_store_tile(const A &a, bool mine, double qi, int lane,
                                               double *__restrict__ vir_tile, int64_t vcap,
                                               double *__restrict__ e_lj, int64_t tile)
{
    if constexpr (A::vir) {
#pragma unroll
        for (int c = 0; c < 6; ++c) {
            const double v = warp_sum(mine ? 0.5 * qi * (double)a.w[c] : 0.0);
            if (lane == 0) vir_tile[c * vcap + tile] = v;
        }
    }
    if constexpr (A::lj) {
        const double v = warp_sum(mine ? 0.5 * (double)a.lj_f[3] : 0.0);
        if (lane == 0) e_lj[tile] = v;
    }
    if constexpr (A::vir && A::lj) {
#pragma unroll
        for (int c = 0; c < 6; ++c) {
            const double v = warp_sum(mine ? 0.5 * (double)a.lj_w[c] : 0.0);
            if (lane == 0) vir_tile[(6 + c) * vcap + tile] = v;
        }
    }
}

// Lennard-Jones arguments of the real-space kernels: sorted types, the [T][T] table of
// (sigma^2, 4 eps, 24 eps, -) and the per-tile energy output.
struct LJArgs {
    const int *tsort;
    const double *tab;
    int ntypes;
    double *e_tile;
};

// Shared-memory copy of the pair table with the shift u(r_c) of every pair type in the
// fourth entry; every thread of the block takes part (call before any thread returns).
template <class T, class T4>
__device__ __forceinline__ void load_lj_table(T4 *ljs, const LJArgs &lj, double rc2)
{
    for (int u = threadIdx.x; u < lj.ntypes * lj.ntypes; u += blockDim.x) {
        const double s2 = lj.tab[4 * u], e4 = lj.tab[4 * u + 1];
        const double x2 = s2 / rc2, x6 = x2 * x2 * x2;
        T4 c;
        c.x = (T)s2;
        c.y = (T)e4;
        c.z = (T)lj.tab[4 * u + 2];
        c.w = (T)(e4 * (x6 * x6 - x6));
        ljs[u] = c;
    }
    __syncthreads();
}

// erfc(x) = exp(-x^2) * t * exp(P(t)), t = 1 / (1 + x / 2), x >= 0: the Chebyshev fit
// "erfcc" of Numerical Recipes in C (2nd ed., Sec. 6.2), fractional error below 1.2e-7 in
// exact arithmetic (checked against the double-precision erfc in tests/test_abi_cpu.py).
// The caller supplies g = exp(-x^2), which the force term needs as well.
__device__ __forceinline__ float erfc_from_gauss(float x, float g)
{
    const float t = __fdividef(1.0f, 1.0f + 0.5f * x);
    float p = 0.17087277f;
    p = fmaf(p, t, -0.82215223f);
    p = fmaf(p, t, 1.48851587f);
    p = fmaf(p, t, -1.13520398f);
    p = fmaf(p, t, 0.27886807f);
    p = fmaf(p, t, -0.18628806f);
    p = fmaf(p, t, 0.09678418f);
    p = fmaf(p, t, 0.37409196f);
    p = fmaf(p, t, 1.00002368f);
    p = fmaf(p, t, -1.26551223f);
    return t * g * __expf(p);
}

// One candidate pair: target at the origin shifted by (xi, yi, zi), partner p; with
// Lennard-Jones pairs, ljrow is the target type's row of the table and tj the partner's type.
template <class T, class T4, class A>
__device__ __forceinline__ void pair(A &a, const T4 &p, T xi, T yi, T zi, T rc2,
                                     T beta, T nb2, T two_b_rpi, const T4 *ljrow, int tj)
{
    const T dx = xi - p.x, dy = yi - p.y, dz = zi - p.z;   // r_i - r_j
    const T r2 = dx * dx + dy * dy + dz * dz;
    if (r2 < rc2 && r2 > T(0)) {
        const T rinv = rsqrt_t(r2);
        const T r = r2 * rinv;
        const T g = exp_t(nb2 * r2);                        // exp(-beta^2 r^2)
        T e;                                                // erfc(beta r) / r
        if constexpr (sizeof(T) == 4) e = erfc_from_gauss(beta * r, g) * rinv;
        else e = erfc_t(beta * r) * rinv;
        const T s = p.w * (e + two_b_rpi * g) * rinv * rinv;
        a.phi += p.w * e;
        const T sx = s * dx, sy = s * dy, sz = s * dz;
        a.fx += sx;
        a.fy += sy;
        a.fz += sz;
        if constexpr (A::vir) {
            a.w[0] += sx * dx; a.w[1] += sy * dy; a.w[2] += sz * dz;
            a.w[3] += sx * dy; a.w[4] += sx * dz; a.w[5] += sy * dz;
        }
        if constexpr (A::lj) {
            // u = 4 eps (x^12 - x^6) - u(r_c), x = sigma / r; -du/dr / r = 24 eps (2 x^12 - x^6) / r^2
            const T4 c = ljrow[tj];
            const T inv2 = rinv * rinv;
            const T x2 = c.x * inv2, x6 = x2 * x2 * x2;
            const T fl = c.z * (T(2) * x6 * x6 - x6) * inv2;
            const T lx = fl * dx, ly = fl * dy, lz = fl * dz;
            a.lj_f[0] += lx;
            a.lj_f[1] += ly;
            a.lj_f[2] += lz;
            a.lj_f[3] += c.y * (x6 * x6 - x6) - c.w;
            if constexpr (A::vir) {
                a.lj_w[0] += lx * dx; a.lj_w[1] += ly * dy; a.lj_w[2] += lz * dz;
                a.lj_w[3] += lx * dy; a.lj_w[4] += lx * dz; a.lj_w[5] += ly * dz;
            }
        }
    }
}

// Chunk of a contiguous run of partner cells staged in shared memory.
struct Chunk {
    int g0, cnt;        // sorted range [g0, g0 + cnt)
    int rowbase;        // nrow * nc
    int u0;             // unwrapped x index of the first cell of the run
    int dy, dz;
};

struct ChunkIter {
    // stencil position
    int dz, dy, w, nc;
    int xa, xb;          // tile x-cell range
    int row_cy, row_cz;
    int wx;              // x reach of the current row
    int u, uend;         // next unwrapped cell to start a run, last cell of the row range
    // current run
    int g, gend, run_u0, rowbase;
    bool in_run;
    bool started;
    int part, split, rowctr;   // this warp takes the kept rows with index % split == part
    float side, rc2;     // geometry for culling (float is enough for the reach test)

    __device__ bool next_row()
    {
        while (true) {
            if (!started) { started = true; dz = -w; dy = -w; }
            else if (++dy > w) { dy = -w; if (++dz > w) return false; }
            int ay = dy < 0 ? -dy : dy, az = dz < 0 ? -dz : dz;
            float my = ay > 0 ? (ay - 1) * side : 0.f, mz = az > 0 ? (az - 1) * side : 0.f;
            float rest = rc2 - my * my - mz * mz;
            if (rest <= 0.f) continue;
            if ((rowctr++ % split) != part) continue;
            int r = (int)ceilf(sqrtf(rest) / side - 1e-6f);
            wx = r < w ? r : w;
            if (wx < 0) wx = 0;
            u = xa - wx;
            uend = xb + wx;
            int ny = ((row_cy + dy) % nc + nc) % nc, nz = ((row_cz + dz) % nc + nc) % nc;
            rowbase = (nz * nc + ny) * nc;
            return true;
        }
    }

    __device__ bool next(const int *__restrict__ cell_start, Chunk &c)
    {
        while (true) {
            if (in_run && g < gend) {
                int cnt = gend - g < kCap ? gend - g : kCap;
                c.g0 = g; c.cnt = cnt; c.rowbase = rowbase; c.u0 = run_u0; c.dy = dy; c.dz = dz;
                g += cnt;
                return true;
            }
            in_run = false;
            if (!started || u > uend) {
                if (!next_row()) return false;
            }
            int c0 = ((u % nc) + nc) % nc;
            int u1 = u + (nc - 1 - c0);
            if (u1 > uend) u1 = uend;
            g = cell_start[rowbase + c0];
            gend = cell_start[rowbase + c0 + (u1 - u) + 1];
            run_u0 = u;
            u = u1 + 1;
            in_run = true;
        }
    }
};

template <class T, int kTile, bool kVir, bool kLJ>
__global__ void __launch_bounds__(kWarps * 32)
k_real_cells(const typename Vec4<T>::type *__restrict__ pl, const int *__restrict__ key_sorted,
             const int *__restrict__ cell_start, const int2 *__restrict__ tiles,
             const int *__restrict__ tile_total, int nc, int w, T side, T rc2, T beta,
             T two_b_rpi, int split, double *__restrict__ f_out, double *__restrict__ phi_out,
             double *__restrict__ e_tile, double *__restrict__ vir_tile, int64_t vcap,
             LJArgs lj, int *__restrict__ status)
{
    using T4 = typename Vec4<T>::type;
    using Acc = PairAcc<T, kVir, kLJ>;
    __shared__ T4 ljs[kLJ ? EWALD_LJ_MAX_TYPES * EWALD_LJ_MAX_TYPES : 1];
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t bars[kWarps][2];
    __shared__ Acc xacc[kWarps][32];            // partial sums handed between split warps
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    T4 *buf[2];
    buf[0] = reinterpret_cast<T4 *>(smem_raw) + (size_t)warp * 2 * kCap;
    buf[1] = buf[0] + kCap;
    uint64_t *bar = bars[warp];
    if (lane == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_mbar_init();
    }
    __syncwarp();
    if constexpr (kLJ) load_lj_table<T, T4>(ljs, lj, (double)rc2);
    // with split = 2 the two warps 2t and 2t + 1 of a block share a tile, each taking every
    // other stencil row; their sums are added (in that order) at the end
    const int part = warp % split;
    const int tile = (blockIdx.x * kWarps + warp) / split;
    const bool active = tile < *tile_total;
    if (split == 1 && !active) return;

    const int2 td = active ? tiles[tile] : make_int2(0, 0);
    const int row = td.x, first = td.y;
    const int row_end = active ? cell_start[(row + 1) * nc] : 1;
    const int last = active ? min(first + kTile, row_end) - 1 : 0;
    constexpr int kGroups = 32 / kTile;             // partner lanes per target
    const int ti = lane % kTile, g = lane / kTile;   // target slot, partner group
    const int i = first + ti;
    const bool valid = i <= last;
    const T4 pi = pl[valid ? i : last];
    const int cxi = key_sorted[valid ? i : last] % nc;
    const T4 *ljrow = kLJ ? ljs + lj.tsort[valid ? i : last] * lj.ntypes : nullptr;

    ChunkIter it;
    it.w = w; it.nc = nc;
    it.xa = key_sorted[first] % nc;
    it.xb = key_sorted[last] % nc;
    it.row_cy = row % nc; it.row_cz = row / nc;
    it.in_run = false; it.started = false;
    it.part = part; it.split = split; it.rowctr = 0;
    it.side = (float)side; it.rc2 = (float)rc2;
    it.u = 0; it.uend = -1;

    Acc acc{};
    const T nb2 = -beta * beta;
    uint32_t phase[2] = {0u, 0u};
    Chunk cur, nxt;
    bool have_cur = active && it.next(cell_start, cur);
    bool ok = true;
    if (have_cur && lane == 0) {
        mbar_expect_tx(&bar[0], cur.cnt * (uint32_t)sizeof(T4));
        tma_bulk_g2s(buf[0], pl + cur.g0, cur.cnt * (uint32_t)sizeof(T4), &bar[0]);
    }
    int b = 0;
    while (have_cur) {
        bool have_nxt = it.next(cell_start, nxt);
        if (have_nxt && lane == 0) {
            // the other buffer was fully read before the last __syncwarp of the loop
            fence_proxy_async();
            mbar_expect_tx(&bar[b ^ 1], nxt.cnt * (uint32_t)sizeof(T4));
            tma_bulk_g2s(buf[b ^ 1], pl + nxt.g0, nxt.cnt * (uint32_t)sizeof(T4), &bar[b ^ 1]);
        }
        if (!warp_wait(&bar[b], phase[b])) { ok = false; break; }
        phase[b] ^= 1u;

        const T yi = pi.y - T(cur.dy) * side;
        const T zi = pi.z - T(cur.dz) * side;
        const T4 *sb = buf[b];
        // walk the cells of the run that overlap [g0, g0 + cnt); inside a run the cell index
        // advances with u without wrapping, and each cell ends where the next one starts
        int u = cur.u0;
        const int cend = cur.g0 + cur.cnt;
        int c = u < 0 ? u + nc : (u >= nc ? u - nc : u);
        const int *cs = cell_start + cur.rowbase;
        int cb = cs[c];
        while (true) {
            const int ce = cs[c + 1];
            if (ce > cur.g0) {
                const int jb = (cb > cur.g0 ? cb : cur.g0) - cur.g0;
                const int je = (ce < cend ? ce : cend) - cur.g0;
                const T xi = pi.x - T(u - cxi) * side;
                for (int j = jb + g; j < je; j += kGroups)
                    pair<T, T4>(acc, sb[j], xi, yi, zi, rc2, beta, nb2, two_b_rpi, ljrow,
                                kLJ ? lj.tsort[cur.g0 + j] : 0);
            }
            if (ce >= cend) break;
            cb = ce;
            ++u;
            ++c;
        }
        __syncwarp();
        cur = nxt;
        have_cur = have_nxt;
        b ^= 1;
    }
    if (!ok) {
        if (lane == 0) atomicOr(status, kStTimeout);
        // let a copy still in flight land before the warp leaves (bounded)
        warp_wait(&bar[b ^ 1], phase[b ^ 1]);
        if (split == 1) return;
    }
    // combine the kGroups partner groups of every target (lanes ti, ti + kTile, ...)
#pragma unroll
    for (int o = kTile; o < 32; o <<= 1) acc_shfl_add(acc, o);
    if (split == 2) {
        // every warp of the block reaches this barrier (none has returned with split = 2)
        if (part == 1) xacc[warp][lane] = acc;
        __syncthreads();
        if (part == 1 || !active) return;
        acc_add(acc, xacc[warp + 1][lane]);
    }
    const double qi = (double)pi.w;
    if (valid && g == 0) {
        double f[3] = {qi * (double)acc.fx, qi * (double)acc.fy, qi * (double)acc.fz};
        if constexpr (kLJ) {
            f[0] += (double)acc.lj_f[0];
            f[1] += (double)acc.lj_f[1];
            f[2] += (double)acc.lj_f[2];
        }
        f_out[3 * (int64_t)i + 0] = f[0];
        f_out[3 * (int64_t)i + 1] = f[1];
        f_out[3 * (int64_t)i + 2] = f[2];
        phi_out[i] = (double)acc.phi;
    }
    const double e = warp_sum((valid && g == 0) ? qi * (double)acc.phi : 0.0);
    if (lane == 0) e_tile[tile] = e;
    acc_store_tile(acc, valid && g == 0, qi, lane, vir_tile, vcap, lj.e_tile, tile);
}

// All pairs with the minimum image (boxes too small for a cell stencil): one tile of 32
// targets per warp, every particle staged through the same double-buffered TMA path.
template <class T, bool kVir, bool kLJ>
__global__ void __launch_bounds__(kWarps * 32)
k_real_allpairs(const typename Vec4<T>::type *__restrict__ pl, int n, T L, T rc2, T beta,
                T two_b_rpi, double *__restrict__ f_out, double *__restrict__ phi_out,
                double *__restrict__ e_tile, double *__restrict__ vir_tile, int64_t vcap,
                LJArgs lj, int *__restrict__ status)
{
    using T4 = typename Vec4<T>::type;
    __shared__ T4 ljs[kLJ ? EWALD_LJ_MAX_TYPES * EWALD_LJ_MAX_TYPES : 1];
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t bars[kWarps][2];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    T4 *buf[2];
    buf[0] = reinterpret_cast<T4 *>(smem_raw) + (size_t)warp * 2 * kCapAll;
    buf[1] = buf[0] + kCapAll;
    uint64_t *bar = bars[warp];
    if (lane == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_mbar_init();
    }
    __syncwarp();
    if constexpr (kLJ) load_lj_table<T, T4>(ljs, lj, (double)rc2);
    const int tile = blockIdx.x * kWarps + warp;
    if (tile * 32 >= n) return;
    const int i = tile * 32 + lane;
    const bool valid = i < n;
    const T4 pi = pl[valid ? i : n - 1];
    const T4 *ljrow = kLJ ? ljs + lj.tsort[valid ? i : n - 1] * lj.ntypes : nullptr;
    const T invL = T(1) / L;
    PairAcc<T, kVir, kLJ> acc{};
    const T nb2 = -beta * beta;
    uint32_t phase[2] = {0u, 0u};
    const int nchunks = (n + kCapAll - 1) / kCapAll;
    if (lane == 0) {
        int cnt = min(kCapAll, n);
        mbar_expect_tx(&bar[0], cnt * (uint32_t)sizeof(T4));
        tma_bulk_g2s(buf[0], pl, cnt * (uint32_t)sizeof(T4), &bar[0]);
    }
    bool ok = true;
    int b = 0;
    for (int c = 0; c < nchunks; ++c) {
        if (c + 1 < nchunks && lane == 0) {
            int g = (c + 1) * kCapAll, cnt = min(kCapAll, n - g);
            fence_proxy_async();
            mbar_expect_tx(&bar[b ^ 1], cnt * (uint32_t)sizeof(T4));
            tma_bulk_g2s(buf[b ^ 1], pl + g, cnt * (uint32_t)sizeof(T4), &bar[b ^ 1]);
        }
        if (!warp_wait(&bar[b], phase[b])) { ok = false; break; }
        phase[b] ^= 1u;
        const int cnt = min(kCapAll, n - c * kCapAll);
        const T4 *sb = buf[b];
        for (int j = 0; j < cnt; ++j) {
            T4 p = sb[j];
            T dx = pi.x - p.x, dy = pi.y - p.y, dz = pi.z - p.z;
            dx -= L * rint(dx * invL);
            dy -= L * rint(dy * invL);
            dz -= L * rint(dz * invL);
            // evaluate the pair at the minimum image: shift the partner, keep the target
            T4 pj = p;
            pj.x = pi.x - dx; pj.y = pi.y - dy; pj.z = pi.z - dz;
            pair<T, T4>(acc, pj, pi.x, pi.y, pi.z, rc2, beta, nb2, two_b_rpi, ljrow,
                        kLJ ? lj.tsort[c * kCapAll + j] : 0);
        }
        __syncwarp();
        b ^= 1;
    }
    if (!ok) {
        if (lane == 0) atomicOr(status, kStTimeout);
        warp_wait(&bar[b ^ 1], phase[b ^ 1]);
        return;
    }
    const double qi = (double)pi.w;
    if (valid) {
        double f[3] = {qi * (double)acc.fx, qi * (double)acc.fy, qi * (double)acc.fz};
        if constexpr (kLJ) {
            f[0] += (double)acc.lj_f[0];
            f[1] += (double)acc.lj_f[1];
            f[2] += (double)acc.lj_f[2];
        }
        f_out[3 * (int64_t)i + 0] = f[0];
        f_out[3 * (int64_t)i + 1] = f[1];
        f_out[3 * (int64_t)i + 2] = f[2];
        phi_out[i] = (double)acc.phi;
    }
    const double e = warp_sum(valid ? qi * (double)acc.phi : 0.0);
    if (lane == 0) e_tile[tile] = e;
    acc_store_tile(acc, valid, qi, lane, vir_tile, vcap, lj.e_tile, tile);
}

template <class T, bool kVir, bool kLJ>
cudaError_t launch_real_t(Plan &p, int64_t n, const typename Vec4<T>::type *pl, cudaStream_t st)
{
    Workspace &ws = p.ws;
    double *vir = kVir ? ws.vir_tile : nullptr;
    const int64_t vcap = real_tile_capacity(p, n);
    LJArgs lj{ws.type_sorted, p.lj_tab_d, p.lj_ntypes, ws.elj_tile};
    const size_t smem = (size_t)kWarps * 2 * (p.w == 0 ? kCapAll : kCap) * sizeof(typename Vec4<T>::type);
    const T beta = (T)p.beta, rc2 = (T)(p.rc * p.rc);
    const T tbr = (T)(2.0 * p.beta / sqrt(kPi));
    cudaError_t e;
    if (p.w == 0) {
        auto kern = k_real_allpairs<T, kVir, kLJ>;
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        int tiles = (int)((n + 31) / 32);
        kern<<<(tiles + kWarps - 1) / kWarps, kWarps * 32, smem, st>>>(
            pl, (int)n, (T)p.L, rc2, beta, tbr, ws.f_real, ws.phi_real, ws.e_tile, vir, vcap, lj,
            p.d_status);
    } else {
        auto kern = p.real_tile == kTileDense ? k_real_cells<T, kTileDense, kVir, kLJ>
                                              : k_real_cells<T, kTileSparse, kVir, kLJ>;
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        int64_t tiles = real_tile_capacity(p, n);
        // two warps per tile when one warp per tile would leave the SMs short of warps
        const int split = tiles < 16 * (int64_t)p.num_sms ? 2 : 1;
        kern<<<(unsigned)((tiles * split + kWarps - 1) / kWarps), kWarps * 32, smem, st>>>(
            pl, ws.key_sorted, ws.cell_start, ws.tiles, ws.tile_off + p.nc * p.nc, p.nc, p.w,
            (T)p.cell_side, rc2, beta, tbr, split, ws.f_real, ws.phi_real, ws.e_tile, vir, vcap,
            lj, p.d_status);
    }
    p.launches += 1;
    return cudaGetLastError();
}

template <class T>
cudaError_t launch_real_p(Plan &p, int64_t n, const typename Vec4<T>::type *pl, cudaStream_t st,
                          bool virial)
{
    const bool lj = p.lj_ntypes > 0;
    if (virial) return lj ? launch_real_t<T, true, true>(p, n, pl, st) : launch_real_t<T, true, false>(p, n, pl, st);
    return lj ? launch_real_t<T, false, true>(p, n, pl, st) : launch_real_t<T, false, false>(p, n, pl, st);
}

}  // namespace

int64_t real_tile_capacity(const Plan &p, int64_t n)
{
    if (p.w == 0) return (n + 31) / 32;
    return n / real_tile_size(p) + (int64_t)p.nc * p.nc + 1;
}

int real_tile_size(const Plan &p) { return p.w == 0 ? 32 : (p.real_tile == kTileDense ? kTileDense : kTileSparse); }

int real_tile_for(int w, double cell_occupancy)
{
    if (w == 0) return 32;
    return cell_occupancy >= 16.0 ? kTileDense : kTileSparse;
}

cudaError_t launch_wait_probe(Plan &p, cudaStream_t st)
{
    k_wait_probe<<<1, 32, 0, st>>>(p.d_status);
    p.last_stream = st;
    return cudaGetLastError();
}

cudaError_t launch_real(Plan &p, int64_t n, cudaStream_t st, bool virial)
{
    if (p.precision == EWALD_FP64) return launch_real_p<double>(p, n, p.ws.pl64, st, virial);
    return launch_real_p<float>(p, n, p.ws.pl32, st, virial);
}

}  // namespace ew
