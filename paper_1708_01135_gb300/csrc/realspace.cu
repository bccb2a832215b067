// Real-space pair sum (hot-path step a4): Section 3.1.1, Eq. 4 and Listing 1.
//
//   phi_i = sum_{j : 0 < |r_ij| < r_c} q_j erfc(beta r_ij) / r_ij
//   F_i   = q_i sum_j q_j (r_ij / r_ij^2) [erfc(beta r_ij) / r_ij
//                                          + 2 beta / sqrt(pi) exp(-beta^2 r_ij^2)]
//   E_real = 1/2 sum_i q_i phi_i            (r_ij = r_i - r_j, minimum image)
//
// GPU design (templated on FP64 and FP32 arithmetic), cell mode:
//   * The box is cut into nc^3 cubic cells of side s ~ max(1.33 rho^-1/3, r_c / 5), sorted
//     by cell key (c_z nc + c_y) nc + c_x, so that every row of cells along x (fixed c_y,
//     c_z) is a contiguous range of the sorted arrays; where the rows are long (w >= 5) the
//     particles of a cell are in x order as well (binning, k_rowsort).
//   * A warp owns up to 32 consecutive sorted targets of one row of cells, one lane each.
//     It visits the rows (c_y + dy, c_z + dz), |dy|, |dz| <= w, in a fixed order.  For each
//     row every target takes its own reach: the distance d from its (y, z) to the row's
//     square gives the x half-width sqrt(r_c^2 - d^2), and its candidates are the particles
//     of the row with x in [x - reach, x + reach]: the cells overlapping that window (one
//     or, where the row wraps, two contiguous ranges), with x-ordered cells cut to the
//     window by two binary searches.  The warp stages the union of its targets' ranges in shared
//     memory (bulk copies on an mbarrier, double-buffered) and every lane searches and
//     walks its own range; the warp runs as many steps as its longest range needs.  This
//     keeps the candidates close to the cutoff sphere of each target (about 1.3 to 1.6 per
//     partner inside r_c) instead of the cutoff sphere of a whole tile of targets.  With
//     few groups of targets per SM, two or four warps share a group, each taking every
//     second or fourth row.
//   * FP32: positions are 32-bit fixed-point fractions of the box (x / L 2^32), so the
//     difference of two of them modulo 2^32 is the minimum-image displacement exactly, at
//     2^-32 L resolution whatever the box size (periodic images are implicit); each component
//     is rounded once, to FP32.  FP64: wrapped global coordinates, with the image shift of a
//     wrapped row or range.
//   * erfc in FP32 is t exp(-x^2) P(u), t = 1 / (1 + p x), u = a t + b, with a degree-8
//     polynomial P fitted to erfc(x) exp(x^2) / t (csrc/fit_erfc.py derives the
//     coefficients): one exp2, one reciprocal and the pair's rsqrt.
//   * Every target's sums are held by its lane (and, with shared groups, combined across the
//     warps in part order); the target's force is written by one lane, and no two threads
//     ever write the same particle (the paper's rule that a loop writes only its own
//     particle, Section 3.2.3, with no atomics); energies are one FP64 partial per warp,
//     summed in order by the finalize step.
// All pairs mode (boxes too small for a stencil of distinct cells): one tile of 32 targets
// per warp, every particle staged through a double-buffered bulk TMA copy (cp.async.bulk,
// completion on an mbarrier) and read by all lanes as a broadcast.
#include <cuda_runtime.h>
#include <stdint.h>

#include "ewald_internal.cuh"

namespace ew {
namespace {

constexpr int kWarps = 4;      // warps (tiles) per block
constexpr int kCapAll = 256;   // particles per staging buffer (all-pairs mode)

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
    if (__all_sync(0xffffffffu, mbar_try_wait(bar, parity))) return true;   // usually landed
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
// FP32 pair arithmetic on the special-function unit directly: the approximate PTX forms with
// subnormal inputs and results flushed to zero (pair distances, Gaussians and erfc values of
// interest are far from the subnormal range, and a flushed Gaussian or erfc term is below
// 1e-38 of the pair's Coulomb term).  One instruction each, no special-case paths.
__device__ __forceinline__ float ex2_ftz(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float rcp_ftz(float x)
{
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float rsqrt_ftz(float x)
{
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float sqrt_ftz(float x)
{
    float y;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
constexpr float kLog2e = 1.4426950408889634f;

// exp(-beta^2 r^2) from nb2l = -beta^2 log2(e) (FP32) or nb2 = -beta^2 (FP64)
__device__ __forceinline__ float gauss_t(float nb2l, float r2) { return ex2_ftz(nb2l * r2); }
__device__ __forceinline__ double gauss_t(double nb2, double r2) { return exp(nb2 * r2); }
__device__ __forceinline__ float rsqrt_t(float x) { return rsqrt_ftz(x); }
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
                                               double *__restrict__ e_lj, int64_t tile,
                                               double vscale = 1.0)
{
    if constexpr (A::vir) {
#pragma unroll
        for (int c = 0; c < 6; ++c) {
            const double v = warp_sum(mine ? 0.5 * qi * vscale * (double)a.w[c] : 0.0);
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
// (s2scale multiplies sigma^2, for kernels that take distances in other units than L.)
template <class T, class T4>
__device__ __forceinline__ void load_lj_table(T4 *ljs, const LJArgs &lj, double rc2,
                                              double s2scale = 1.0)
{
    for (int u = threadIdx.x; u < lj.ntypes * lj.ntypes; u += blockDim.x) {
        const double s2 = lj.tab[4 * u], e4 = lj.tab[4 * u + 1];
        const double x2 = s2 / rc2, x6 = x2 * x2 * x2;
        T4 c;
        c.x = (T)(s2 * s2scale);
        c.y = (T)e4;
        c.z = (T)lj.tab[4 * u + 2];
        c.w = (T)(e4 * (x6 * x6 - x6));
        ljs[u] = c;
    }
    __syncthreads();
}

// erfc(x) ~= t exp(-x^2) P(u), t = 1 / (1 + p x), u = a t + b, x >= 0: a degree-8 polynomial
// fitted to erfc(x) exp(x^2) / t on [0, 8] (csrc/fit_erfc.py: relative error 7.6e-9 in exact
// arithmetic with the coefficients kErfcC + kErfcCL, 3.5e-7 with kErfcC and FP32 rounding of
// t, u and the Horner steps).  Beyond x = 8, where
// erfc < 1e-29, the polynomial is extrapolated; those pairs add nothing measurable.  The
// caller supplies g = exp(-x^2), which the force term needs as well.
constexpr float kErfcP = 0.3700000047683716f;
constexpr float kErfcA = 2.675675630569458f, kErfcB = -1.675675630569458f;
__constant__ float kErfcC[9] = {0.48547884821891785f, 0.31732580065727234f, 0.14685595035552979f,
                             0.044840894639492035f, 0.006656187120825052f,
                             -0.0007446469971910119f, -0.000444741832325235f,
                             7.326919330807868e-06f, 2.438715091557242e-05f};
// FP32 remainders of the fitted coefficients (the double-float near-pair path)
__constant__ float kErfcCL[9] = {-3.958085414978996e-09f, -4.999006097961001e-09f,
                              7.110552147082672e-10f, -1.6942547365061955e-09f,
                              1.4456411068231034e-10f, 1.9717394383889086e-11f,
                              4.030599205090413e-12f, -2.7720381396670497e-14f,
                              8.240692741905142e-13f};

__device__ __forceinline__ float erfc_from_gauss(float x, float g)
{
    const float t = rcp_ftz(fmaf(kErfcP, x, 1.0f));
    const float u = fmaf(kErfcA, t, kErfcB);
    float p = kErfcC[8];
#pragma unroll
    for (int k = 7; k >= 0; --k) p = fmaf(p, u, kErfcC[k]);
    return t * g * p;
}

// One candidate pair with displacement d = r_i - r_j (minimum image) and partner charge qj;
// the pair counts when 0 < |d| < r_c.  nb2 is -beta^2 log2(e) in FP32, -beta^2 in FP64 (see
// gauss_t).  With Lennard-Jones pairs, ljrow is the target type's row of the table and tj
// the partner's type.
template <class T, class T4, class A>
__device__ __forceinline__ void pair_d(A &a, T dx, T dy, T dz, T qj, T rc2, T beta, T nb2,
                                       T two_b_rpi, const T4 *ljrow, int tj)
{
    const T r2 = dx * dx + dy * dy + dz * dz;
    if (r2 < rc2 && r2 > T(0)) {
        const T rinv = rsqrt_t(r2);
        const T r = r2 * rinv;
        const T g = gauss_t(nb2, r2);                       // exp(-beta^2 r^2)
        T e;                                                // erfc(beta r) / r
        if constexpr (sizeof(T) == 4) e = erfc_from_gauss(beta * r, g) * rinv;
        else e = erfc_t(beta * r) * rinv;
        const T s = qj * (e + two_b_rpi * g) * rinv * rinv;
        a.phi += qj * e;
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

// The same with the target at (xi, yi, zi) and the partner's position in p.
template <class T, class T4, class A>
__device__ __forceinline__ void pair(A &a, const T4 &p, T xi, T yi, T zi, T rc2,
                                     T beta, T nb2, T two_b_rpi, const T4 *ljrow, int tj)
{
    pair_d<T, T4>(a, xi - p.x, yi - p.y, zi - p.z, p.w, rc2, beta, nb2, two_b_rpi, ljrow, tj);
}

// ---- FP32 pairs in fixed-point units ----------------------------------------------------
//
// The FP32 cell kernel works in units of the fixed-point step S = L / 2^32: a displacement
// component is the integer difference D of two fractions, h = float(D) (rounded once), and
// r^2, beta, the cutoff and the constants are all expressed in these units, so that no
// product with S rounds the geometry.  The accumulated sums are rescaled once per target, in
// FP64 (forces by 1 / S^2, potentials, the Coulomb virial and the Lennard-Jones force by
// 1 / S).
//
// Near pairs (r below r_near, a few mean particle spacings) carry most of the pair forces
// on an ion, and in ionic systems the net force is a small sum of large pair forces.  Two
// treatments (the plan's near-pair mode):
//   * FP32 (default): the pair in FP32 with the exact r^2.  The FP32 r^2 of the rounded
//     components is off by ~2^-24, which alone gives about 1e-6 of the RMS force in a
//     rock-salt crystal; so the exact r^2 = sum D^2 is formed as an FP32 pair (hi + lo):
//     D = h + l with l = D - int(h) exact, h^2 = P + e with e = fma(h, h, -P), and TwoSum
//     errors of the sums; the force factor A = (erfc(beta r)/r + c g)/r^2 and the potential
//     e = erfc(beta r)/r are then corrected to first order in delta = r^2_exact - r^2:
//       dA/d(r^2) = -(1.5 A + c beta^2 g) / r^2,   de/d(r^2) = -(e + c g) / (2 r^2),
//     c = 2 beta / sqrt(pi), g = exp(-beta^2 r^2) (delta / r^2 is ~2^-24, so the second
//     order is ~2^-48).  What remains is the FP32 rounding of the special functions and of
//     the products, ~1e-7 of every pair.
//   * double-float (kDF): the near pairs leave pair_s and are evaluated in double-float
//     arithmetic (near_term), ~1e-8 of every pair, at the cost of a second scan of the
//     staged candidates within r_near.
// The split is taken on the FP32 r^2 of the rounded components in both passes, so every pair
// is counted once.
struct ScaledK {
    float rc2s, rn2s;       // r_c^2 and r_near^2 in units of S^2
    float beta_s;           // beta S
    float nb2l_s;           // -beta^2 S^2 log2(e)
    float c_s;              // 2 beta / sqrt(pi) S
    float cb2_s;            // c_s beta_s^2
};

// Double-float constants of the near pairs (value = h + l).
struct NearK {
    float beta_h, beta_l;   // beta S
    float c_h, c_l;         // 2 beta / sqrt(pi) S
    float rn2m;             // r_near^2 (physical units) with the range margin
};

__device__ __forceinline__ float r2_f32(float hx, float hy, float hz)
{
    return fmaf(hx, hx, fmaf(hy, hy, hz * hz));
}

__device__ __forceinline__ void two_sum(float a, float b, float &s, float &err)
{
    s = a + b;
    const float bb = s - a;
    err = (a - (s - bb)) + (b - bb);
}

// Residual delta = (exact sum of D_a^2) - r2 for the rounded components h_a = float(D_a),
// r2 being the FP32 value the pair was evaluated at.
__device__ __forceinline__ float r2_residual(int Dx, int Dy, int Dz, float hx, float hy,
                                             float hz, float r2)
{
    const float lx = (float)(Dx - __float2int_rn(hx));
    const float ly = (float)(Dy - __float2int_rn(hy));
    const float lz = (float)(Dz - __float2int_rn(hz));
    const float px = hx * hx, py = hy * hy, pz = hz * hz;
    const float ex = fmaf(hx, hx, -px), ey = fmaf(hy, hy, -py), ez = fmaf(hz, hz, -pz);
    float s1, t1, s2, t2;
    two_sum(px, py, s1, t1);
    two_sum(s1, pz, s2, t2);
    const float cross = fmaf(2.0f * hx, lx, lx * lx) + fmaf(2.0f * hy, ly, ly * ly) +
                        fmaf(2.0f * hz, lz, lz * lz);
    return (s2 - r2) + ((t1 + t2) + ((ex + ey + ez) + cross));
}

// One candidate of the FP32 pass.  Coulomb: 0 < r < r_c, with the first-order r^2 correction
// below r_near; with kDF, r_near <= r < r_c only.  Lennard-Jones: 0 < r < r_c.
template <bool kDF, class T4, class A>
__device__ __forceinline__ void pair_s(A &a, int Dx, int Dy, int Dz, float qj, const ScaledK &K,
                                       const T4 *ljrow, int tj)
{
    const float hx = (float)Dx, hy = (float)Dy, hz = (float)Dz;
    const float r2 = r2_f32(hx, hy, hz);
    const bool coul = kDF ? (r2 < K.rc2s && r2 >= K.rn2s) : (r2 < K.rc2s && r2 > 0.0f);
    if ((kDF && A::lj) ? (r2 < K.rc2s && r2 > 0.0f) : coul) {
        const float rinv = rsqrt_ftz(r2);
        const float rinv2 = rinv * rinv;
        if (!(kDF && A::lj) || coul) {
            const float r = r2 * rinv;
            const float g = ex2_ftz(K.nb2l_s * r2);
            float e = erfc_from_gauss(K.beta_s * r, g) * rinv;
            float fA = fmaf(K.c_s, g, e) * rinv2;
            if constexpr (!kDF) {
                if (r2 < K.rn2s) {
                    const float rho = r2_residual(Dx, Dy, Dz, hx, hy, hz, r2) * rinv2;
                    fA = fmaf(-fmaf(1.5f, fA, K.cb2_s * g), rho, fA);
                    e = fmaf(-0.5f * fmaf(K.c_s, g, e), rho, e);
                }
            }
            const float s = qj * fA;
            a.phi += qj * e;
            const float sx = s * hx, sy = s * hy, sz = s * hz;
            a.fx += sx;
            a.fy += sy;
            a.fz += sz;
            if constexpr (A::vir) {
                a.w[0] += sx * hx; a.w[1] += sy * hy; a.w[2] += sz * hz;
                a.w[3] += sx * hy; a.w[4] += sx * hz; a.w[5] += sy * hz;
            }
        }
        if constexpr (A::lj) {
            // the pair table holds sigma^2 in units of S^2 (load_lj_table's scale)
            const T4 c = ljrow[tj];
            const float x2 = c.x * rinv2, x6 = x2 * x2 * x2;
            const float fl = c.z * (2.0f * x6 * x6 - x6) * rinv2;
            const float lx = fl * hx, ly = fl * hy, lz = fl * hz;
            a.lj_f[0] += lx;
            a.lj_f[1] += ly;
            a.lj_f[2] += lz;
            a.lj_f[3] += c.y * (x6 * x6 - x6) - c.w;
            if constexpr (A::vir) {
                a.lj_w[0] += lx * hx; a.lj_w[1] += ly * hy; a.lj_w[2] += lz * hz;
                a.lj_w[3] += lx * hy; a.lj_w[4] += lx * hz; a.lj_w[5] += ly * hz;
            }
        }
    }
}

// ---- double-float arithmetic: a value is the unevaluated sum h + l of two FP32 numbers -----
// (Dekker's and Knuth's error-free transformations: TwoSum, and TwoProduct with an FMA.)
struct df { float h, l; };

__device__ __forceinline__ df df_fast(float a, float b)     // |a| >= |b|
{
    const float s = a + b;
    return {s, b - (s - a)};
}
__device__ __forceinline__ df df_sum(float a, float b)
{
    const float s = a + b, bb = s - a;
    return {s, (a - (s - bb)) + (b - bb)};
}
__device__ __forceinline__ df df_prod(float a, float b)
{
    const float p = a * b;
    return {p, fmaf(a, b, -p)};
}
__device__ __forceinline__ df df_add(df a, df b)
{
    const df s = df_sum(a.h, b.h);
    return df_fast(s.h, s.l + (a.l + b.l));
}
__device__ __forceinline__ df df_mul(df a, df b)
{
    const df p = df_prod(a.h, b.h);
    return df_fast(p.h, fmaf(a.h, b.l, fmaf(a.l, b.h, p.l)));
}
__device__ __forceinline__ df df_mulf(df a, float b)
{
    const df p = df_prod(a.h, b);
    return df_fast(p.h, fmaf(a.l, b, p.l));
}
__device__ __forceinline__ df df_from_int(int v)
{
    const float h = (float)v;
    return {h, (float)(v - __float2int_rn(h))};
}

// 2^(j/64), j = 0..63, as double-float pairs (filled once per block from FP64 exp2)
__device__ __forceinline__ void load_exp2_table(float2 *tab)
{
    for (int j = threadIdx.x; j < 64; j += blockDim.x) {
        const double v = exp2((double)j / 64.0);
        const float h = (float)v;
        tab[j] = make_float2(h, (float)(v - (double)h));
    }
}

// exp(-x^2) for a double-float x, 0 <= x < 9: 2^y with y = -x^2 log2(e) in double-float,
// y = (64 m + j + f) / 64 with |f| <= 1/2, 2^(j/64) from the table and
// 2^(f/64) - 1 = w (1 + w/2 + w^2/6 + w^3/24), w = f ln2 / 64 (|w| < 0.0055, the series'
// remainder < 4e-14).
__device__ __forceinline__ df gauss_df(df x, const float2 *tab)
{
    const df x2 = df_mul(x, x);
    // -log2(e) = -(1.4426950 + 1.9259630e-8) in double-float
    const df y = df_mul(x2, df{-1.44269502162933349609375f, -1.925963033500011079e-8f});
    const float zh = y.h * 64.0f, zl = y.l * 64.0f;          // exact scalings
    const float nz = rintf(zh);
    const float f = (zh - nz) + zl;                          // zh - nz is exact
    const int n = (int)nz;
    const int j = n & 63, m = (n - j) >> 6;                  // n = 64 m + j, 0 <= j < 64
    const float w = f * 0.010830424696249145f;               // ln(2) / 64
    const float d = w * fmaf(w, fmaf(w, fmaf(w, 0.041666666666666664f, 0.16666666666666666f), 0.5f), 1.0f);
    const float2 t = tab[j];
    df g = df_fast(t.x, fmaf(t.x, d, t.y));
    const float sc = __int_as_float((127 + m) << 23);        // 2^m, m >= -117 for x < 9
    g.h *= sc;
    g.l *= sc;
    return g;
}

// Terms of one near pair: force components and potential (double-float), virial (FP32).
template <bool kVir> struct NearTerm {
    df fx{0.f, 0.f}, fy{0.f, 0.f}, fz{0.f, 0.f}, phi{0.f, 0.f};
    float w[kVir ? 6 : 1] = {};
};

// The Coulomb terms of a near pair (0 < r < r_near) in double-float arithmetic, from the
// integer displacement D (units of S) and the partner charge qj.
template <bool kVir>
__device__ __forceinline__ NearTerm<kVir> near_term(int Dx, int Dy, int Dz, float qj,
                                                    const NearK &N, const float2 *tab)
{
    // D = h + l exactly; r^2 = sum h^2 + sum (2 h l + l^2), the first sum with its rounding
    // errors (|l| <= 128, so the second sum is ~2^-23 of r^2 and its own rounding negligible)
    const df dx = df_from_int(Dx), dy = df_from_int(Dy), dz = df_from_int(Dz);
    const df px = df_prod(dx.h, dx.h), py = df_prod(dy.h, dy.h), pz = df_prod(dz.h, dz.h);
    const df s1 = df_sum(px.h, py.h), s2 = df_sum(s1.h, pz.h);
    const float cross = fmaf(2.0f * dx.h, dx.l, dx.l * dx.l) + fmaf(2.0f * dy.h, dy.l, dy.l * dy.l) +
                        fmaf(2.0f * dz.h, dz.l, dz.l * dz.l);
    const df r2 = df_fast(s2.h, (s1.l + s2.l) + ((px.l + py.l + pz.l) + cross));
    // 1 / r: the FP32 estimate y and one Newton step on the double-float residual
    // e = 1 - r^2 y^2 (1 / r = y (1 + e / 2), the neglected term is 3 e^2 / 8 ~ 2^-44)
    const float y = rsqrt_ftz(r2.h);
    const df y2 = df_prod(y, y);
    const df p = df_prod(r2.h, y2.h);
    const float res = ((1.0f - p.h) - p.l) - fmaf(r2.h, y2.l, r2.l * y2.h);
    const df rinv = df_fast(y, 0.5f * y * res);
    const df rinv2 = df_mul(rinv, rinv);
    const df x = df_mul(df{N.beta_h, N.beta_l}, df_mul(r2, rinv));   // beta r
    const df g = gauss_df(x, tab);                                   // exp(-beta^2 r^2)
    // erfc(x) = t g P(a t + b), t = 1 / (1 + p x)
    const df pxp = df_prod(kErfcP, x.h);
    df dd = df_sum(1.0f, pxp.h);
    dd = df_fast(dd.h, dd.l + (pxp.l + kErfcP * x.l));
    const float th = rcp_ftz(dd.h);
    const float et = fmaf(-th, dd.l, fmaf(-th, dd.h, 1.0f));  // 1 - d th
    const df t = df_fast(th, th * et);
    const df u = df_add(df_mulf(t, kErfcA), df{kErfcB, 0.0f});
    // Horner: the small high-order terms (k >= 4) in FP32, the rest in double-float
    float q = kErfcC[8];
#pragma unroll
    for (int k = 7; k >= 4; --k) q = fmaf(q, u.h, kErfcC[k]);
    df P = df_fast(q, 0.0f);
#pragma unroll
    for (int k = 3; k >= 0; --k) P = df_add(df_mul(P, u), df{kErfcC[k], kErfcCL[k]});
    const df e = df_mul(df_mul(df_mul(t, P), g), rinv);     // erfc(beta r) / r
    const df A = df_mul(df_add(e, df_mul(df{N.c_h, N.c_l}, g)), rinv2);
    const df sq = df_mulf(A, qj);
    NearTerm<kVir> o;
    o.fx = df_mul(sq, dx);
    o.fy = df_mul(sq, dy);
    o.fz = df_mul(sq, dz);
    o.phi = df_mulf(e, qj);
    if constexpr (kVir) {
        o.w[0] = o.fx.h * dx.h; o.w[1] = o.fy.h * dy.h; o.w[2] = o.fz.h * dz.h;
        o.w[3] = o.fx.h * dy.h; o.w[4] = o.fx.h * dz.h; o.w[5] = o.fy.h * dz.h;
    }
    return o;
}

template <bool kVir>
__device__ __forceinline__ void near_add(NearTerm<kVir> &a, const NearTerm<kVir> &o)
{
    a.fx = df_add(a.fx, o.fx);
    a.fy = df_add(a.fy, o.fy);
    a.fz = df_add(a.fz, o.fz);
    a.phi = df_add(a.phi, o.phi);
    if constexpr (kVir) {
#pragma unroll
        for (int c = 0; c < 6; ++c) a.w[c] += o.w[c];
    }
}

template <bool kVir>
__device__ __forceinline__ NearTerm<kVir> near_shfl(const NearTerm<kVir> &v, int src)
{
    NearTerm<kVir> o;
    o.fx = {__shfl_sync(0xffffffffu, v.fx.h, src), __shfl_sync(0xffffffffu, v.fx.l, src)};
    o.fy = {__shfl_sync(0xffffffffu, v.fy.h, src), __shfl_sync(0xffffffffu, v.fy.l, src)};
    o.fz = {__shfl_sync(0xffffffffu, v.fz.h, src), __shfl_sync(0xffffffffu, v.fz.l, src)};
    o.phi = {__shfl_sync(0xffffffffu, v.phi.h, src), __shfl_sync(0xffffffffu, v.phi.l, src)};
    if constexpr (kVir) {
#pragma unroll
        for (int c = 0; c < 6; ++c) o.w[c] = __shfl_sync(0xffffffffu, v.w[c], src);
    }
    return o;
}

// Evaluate the first cnt (<= 32) queued near pairs of a warp, one per lane, and add every
// target's terms into its lane's sums: the entries of one target are added in queue order
// by the first lane that holds one of them, and that sum is passed to the target's lane.
// (ldr: 32 ints of shared memory per warp.)  Whole warp.
template <bool kVir>
__device__ __noinline__ void near_flush(NearTerm<kVir> &acc, const int4 *qd, const int *qt,
                                           int *ldr, int cnt, int lane, const NearK &N,
                                           const float2 *tab)
{
    const bool has = lane < cnt;
    const int tgt = has ? qt[lane] : -1 - lane;      // lanes without an entry: own groups
    NearTerm<kVir> v;
    if (has) {
        const int4 e = qd[lane];
        v = near_term<kVir>(e.x, e.y, e.z, __int_as_float(e.w), N, tab);
    }
    const unsigned grp = __match_any_sync(0xffffffffu, tgt);
    const bool leader = (grp & ((1u << lane) - 1u)) == 0u;
    const int rounds = __reduce_max_sync(0xffffffffu, __popc(grp));
    // the leader adds its group's later entries into its own terms (a leader's terms are
    // never read by another group, a member's only by its leader, before any change)
    unsigned rest = grp & (grp - 1u);
    for (int k = 1; k < rounds; ++k) {
        const int src = rest ? __ffs(rest) - 1 : lane;
        const NearTerm<kVir> o = near_shfl<kVir>(v, src);
        if (leader && rest) near_add<kVir>(v, o);
        rest &= rest - 1u;
    }
    ldr[lane] = -1;
    __syncwarp();
    if (has && leader) ldr[tgt] = lane;
    __syncwarp();
    const int from = ldr[lane];
    const NearTerm<kVir> o = near_shfl<kVir>(v, from >= 0 ? from : lane);
    if (from >= 0) near_add<kVir>(acc, o);
    __syncwarp();
}

// Compensated (Kahan) addition of the row sums of the forces and potential into the totals;
// the other sums are added plainly.
__device__ __forceinline__ void kahan1(float &sum, float &comp, float v)
{
    const float y = v - comp;
    const float t = sum + y;
    comp = (t - sum) - y;
    sum = t;
}
__device__ __forceinline__ void kahan1(double &sum, double &, double v) { sum += v; }
template <class A>
__device__ __forceinline__ void acc_add_rows(A &tot, A &comp, const A &row)
{
    kahan1(tot.fx, comp.fx, row.fx);
    kahan1(tot.fy, comp.fy, row.fy);
    kahan1(tot.fz, comp.fz, row.fz);
    kahan1(tot.phi, comp.phi, row.phi);
    if constexpr (A::vir) {
#pragma unroll
        for (int c = 0; c < 6; ++c) tot.w[c] += row.w[c];
    }
    if constexpr (A::lj) {
#pragma unroll
        for (int c = 0; c < 4; ++c) tot.lj_f[c] += row.lj_f[c];
    }
    if constexpr (A::vir && A::lj) {
#pragma unroll
        for (int c = 0; c < 6; ++c) tot.lj_w[c] += row.lj_w[c];
    }
}

// ---- cell mode: per-target row ranges --------------------------------------------------

// Candidate records of the cell kernel.  FP32: the 32-bit fixed-point fractions x / L, y / L,
// z / L and the bits of q (the sorted copy pu): the difference of two fractions modulo 2^32 is
// the minimum-image displacement exactly, at 2^-32 L resolution, so the only rounding of a
// displacement component is its conversion to FP32 (2^-24 relative).  (Cell-local FP32
// coordinates would carry an absolute error of 2^-24 of the cell side in every stored
// position and in every row offset; for ionic crystals, where the net force is a small sum
// of large pair forces, that doubles the relative force error.)  FP64: the wrapped global
// position and q (the sorted copy pg).
template <class T> struct RowRec;
template <> struct RowRec<float> { using type = uint4; };
template <> struct RowRec<double> { using type = double4_32a; };

__device__ __forceinline__ float rec_q(const uint4 &p) { return __uint_as_float(p.w); }
__device__ __forceinline__ double rec_q(const double4_32a &p) { return p.w; }

// Staged union of the targets' ranges in one row: unwrapped cell bins [A0, A1] of the row,
// laid out in shared memory in bin order as up to three contiguous runs of the sorted array:
// part A, the bins below 0 (the far end of the row, wrapped), part B, the bins inside the
// row, part C, the bins at or beyond nc (the start of the row, wrapped).
struct RowUnion {
    int sA, lenA, sB, lenB, sC, lenC;
    __device__ int total() const { return lenA + lenB + lenC; }
};

// Offset in the staged union of the first particle of unwrapped bin b (A0 <= b <= A1 + 1).
__device__ __forceinline__ int union_off(const RowUnion &u, const int *__restrict__ cs, int nc,
                                         int b)
{
    if (b < 0) return cs[b + nc] - u.sA;
    if (b < nc) return u.lenA + cs[b] - u.sB;
    return u.lenA + u.lenB + cs[b - nc] - u.sC;
}

// One staged item: a chunk [c0, c0 + cnt) of the union of row (dy, dz), and this target's
// range [off0, off1) in the union.
struct RowItem {
    int dy, dz;
    RowUnion u;
    int c0, cnt;
    int off0, off1;
    int noff0, noff1;           // this target's near range (reach r_near) in the union
    // x window (x-ordered cells): the candidates of [off0, off1) whose x displacement lies
    // outside [-xr, xr] are cut off; xr = 0: no cut
    int xr;
};

// Issue the bulk copies of an item into dst (lane 0 only): the parts of the union that the
// chunk overlaps, one mbarrier for all of them.
template <class R4>
__device__ __forceinline__ void issue_item(const RowItem &it, const R4 *__restrict__ pr,
                                           R4 *dst, uint64_t *bar)
{
    mbar_expect_tx(bar, it.cnt * (uint32_t)sizeof(R4));
    const int e = it.c0 + it.cnt;
    const int pb[3] = {0, it.u.lenA, it.u.lenA + it.u.lenB};
    const int pe[3] = {it.u.lenA, it.u.lenA + it.u.lenB, it.u.total()};
    const int ps[3] = {it.u.sA, it.u.sB, it.u.sC};
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const int lo = it.c0 > pb[k] ? it.c0 : pb[k];
        const int hi = e < pe[k] ? e : pe[k];
        if (hi > lo)
            tma_bulk_g2s(dst + (lo - it.c0), pr + ps[k] + (lo - pb[k]),
                         (uint32_t)(hi - lo) * (uint32_t)sizeof(R4), bar);
    }
}

// First g in [lo, hi) whose x displacement (int)(ux - sb[g].x) is at most R, or hi; the
// displacements do not increase along [lo, hi) (staged records in x order).
__device__ __forceinline__ int first_within(const uint4 *sb, int lo, int hi, unsigned ux, int R)
{
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if ((int)(ux - sb[mid].x) <= R) hi = mid;
        else lo = mid + 1;
    }
    return lo;
}

// Walks the rows of the stencil (and the chunks of each row's union) of one warp.
struct RowWalk {
    int w, nc, part, split;
    int cx, cy, cz;             // this target's cell
    float xl, yl, zl;           // this target's position inside its cell
    float sidef, inv_side, rc2m;
    float rn2m;                 // r_near^2 with the margin (0: no near ranges)
    bool valid;
    const int *__restrict__ cell_start;
    // position in the stencil
    int dy, dz, rowctr;
    bool started;
    // the current row's union and this target's range, and the next chunk start
    RowItem row;
    int next_c0;
    bool in_row;

    // Next row with a non-empty union; false at the end of the stencil.  x windows (every
    // cell ordered by x): xw on, to_s the scale from length to fixed-point units.
    __device__ bool next_row(bool xw, float to_s)
    {
        while (true) {
            if (!started) { started = true; dz = -w; dy = -w; }
            else if (++dy > w) { dy = -w; if (++dz > w) return false; }
            const int ay = dy < 0 ? -dy : dy, az = dz < 0 ? -dz : dz;
            const float my = ay > 0 ? (ay - 1) * sidef : 0.f, mz = az > 0 ? (az - 1) * sidef : 0.f;
            if (my * my + mz * mz >= rc2m) continue;          // no point of the row in reach
            if ((rowctr++ % split) != part) continue;
            // this target's reach along the row: distance from (y, z) to the row's square
            const float gy = dy > 0 ? dy * sidef - yl : (dy < 0 ? yl - (dy + 1) * sidef : 0.f);
            const float gz = dz > 0 ? dz * sidef - zl : (dz < 0 ? zl - (dz + 1) * sidef : 0.f);
            const float d2 = gy * gy + gz * gz;
            int a0 = 1 << 30, a1 = -(1 << 30), n0 = 1 << 30, n1 = -(1 << 30);
            float reach = 0.f;
            if (valid && d2 < rc2m) {
                // (approximate square root: a relative error of 2^-22 is inside the margin)
                reach = sqrt_ftz(rc2m - d2);
                int b0 = __float2int_rd((xl - reach) * inv_side);
                int b1 = __float2int_rd((xl + reach) * inv_side);
                b0 = b0 < -w ? -w : b0;
                b1 = b1 > w ? w : b1;
                a0 = cx + b0;
                a1 = cx + b1;
                if (d2 < rn2m) {
                    const float rn = sqrt_ftz(rn2m - d2);
                    int e0 = __float2int_rd((xl - rn) * inv_side);
                    int e1 = __float2int_rd((xl + rn) * inv_side);
                    n0 = cx + (e0 < b0 ? b0 : e0);
                    n1 = cx + (e1 > b1 ? b1 : e1);
                }
            }
            const int A0 = __reduce_min_sync(0xffffffffu, a0);
            const int A1 = __reduce_max_sync(0xffffffffu, a1);
            if (A0 > A1) continue;                              // no target reaches the row
            const int uy = cy + dy < 0 ? cy + dy + nc : (cy + dy >= nc ? cy + dy - nc : cy + dy);
            const int uz = cz + dz < 0 ? cz + dz + nc : (cz + dz >= nc ? cz + dz - nc : cz + dz);
            const int *cs = cell_start + (uz * nc + uy) * nc;
            RowUnion &u = row.u;
            u.sA = 0; u.lenA = 0; u.sC = 0; u.lenC = 0;
            if (A0 < 0) { u.sA = cs[A0 + nc]; u.lenA = cs[nc] - u.sA; }
            const int b0 = A0 > 0 ? A0 : 0, b1 = A1 < nc - 1 ? A1 : nc - 1;
            u.sB = cs[b0];
            u.lenB = cs[b1 + 1] - u.sB;
            if (A1 >= nc) { u.sC = cs[0]; u.lenC = cs[A1 - nc + 1] - u.sC; }
            if (u.total() == 0) continue;
            row.dy = dy;
            row.dz = dz;
            row.xr = 0;
            if (a0 <= a1) {
                row.off0 = union_off(u, cs, nc, a0);
                row.off1 = union_off(u, cs, nc, a1 + 1);
                // the target's own x window [x - reach, x + reach] (in fixed-point units,
                // rounded up): candidates beyond it (r above the reach radius, which the
                // pair test would reject too) are cut off when the staged chunk is walked
                if (xw) row.xr = __float2int_ru(reach * to_s) + 1;
            } else {
                row.off0 = row.off1 = 0;
            }
            if (n0 <= n1) {
                row.noff0 = union_off(u, cs, nc, n0);
                row.noff1 = union_off(u, cs, nc, n1 + 1);
            } else {
                row.noff0 = row.noff1 = 0;
            }
            return true;
        }
    }

    template <int kCapR>
    __device__ bool next(RowItem &it, bool xw, float to_s)
    {
        if (!in_row || next_c0 >= row.u.total()) {
            if (!next_row(xw, to_s)) return false;
            in_row = true;
            next_c0 = 0;
        }
        it = row;
        it.c0 = next_c0;
        const int rest = row.u.total() - next_c0;
        it.cnt = rest < kCapR ? rest : kCapR;
        next_c0 += it.cnt;
        return true;
    }
};

template <class T, int G, bool kVir, bool kLJ, bool kDF>
__global__ void __launch_bounds__(kWarps * 32, sizeof(T) == 4 && !kVir && !kLJ ? (kDF ? 6 : 7) : 1)
k_real_rows(const typename RowRec<T>::type *__restrict__ pr, const double4_32a *__restrict__ pg,
            const int *__restrict__ key_sorted, const int *__restrict__ cell_start,
            const int2 *__restrict__ tiles, const int *__restrict__ tile_total, int n,
            int nc, int w, double side_d, double L_d, T rc2, T beta, T two_b_rpi, ScaledK K,
            NearK NK, double inv_s, int split, int xwin, const int *__restrict__ unordered,
            double *__restrict__ f_out, double *__restrict__ phi_out, double *__restrict__ e_tile,
            double *__restrict__ vir_tile, int64_t vcap, LJArgs lj, int *__restrict__ status)
{
    using R4 = typename RowRec<T>::type;
    using T4 = typename Vec4<T>::type;
    using Acc = PairAcc<T, kVir, kLJ>;
    constexpr bool kFP32 = sizeof(T) == 4;
    constexpr bool kNear = kFP32 && kDF;          // near pairs in double-float
    constexpr int kCapR = 3072 / (int)sizeof(R4);  // records per staging buffer (3 KB)
    __shared__ T4 ljs[kLJ ? EWALD_LJ_MAX_TYPES * EWALD_LJ_MAX_TYPES : 1];
    __shared__ Acc xacc[kWarps][32];             // partial sums handed between split warps
    __shared__ double4_32a xsum[kFP32 ? kWarps : 1][32];   // (the Coulomb sums, FP32 kernel)
    __shared__ float2 ex2tab[kNear ? 64 : 1];
    // near-pair queue of every warp: (D, q bits) and target lane, up to 63 entries; group
    // leaders of a flush
    __shared__ int4 nq_d[kNear ? kWarps : 1][kNear ? 64 : 1];
    __shared__ int nq_t[kNear ? kWarps : 1][kNear ? 64 : 1];
    __shared__ int nq_l[kNear ? kWarps : 1][kNear ? 32 : 1];
    __shared__ __align__(128) R4 stage[kWarps][2][kCapR];
    __shared__ __align__(8) uint64_t bars[kWarps][2];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    uint64_t *bar = bars[warp];
    if (lane == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_mbar_init();
    }
    if constexpr (kNear) load_exp2_table(ex2tab);
    __syncthreads();
    // (FP32: sigma^2 in units of S^2, S = inv_s^-1 the fixed-point step)
    if constexpr (kLJ) load_lj_table<T, T4>(ljs, lj, (double)rc2, kFP32 ? inv_s * inv_s : 1.0);
    // with split = 2 or 4 the warps of a block share groups of targets (warps 2t, 2t + 1 or
    // all four), each taking every split-th row of the stencil; their sums are added in that
    // order at the end
    const int part = warp % split;
    const int grp = (blockIdx.x * kWarps + warp) / split;   // tile of this warp
    const int t = lane / G, g = lane % G;
    const bool active = grp < *tile_total;
    if (split == 1 && !active) return;
    // the tile's targets: up to TG consecutive sorted particles of one row of cells
    const int2 td = active ? tiles[grp] : make_int2(0, 0);
    const int row_end = active ? cell_start[(td.x + 1) * nc] : 1;
    const int i = td.y + t;
    const bool valid = active && i < row_end;
    const int ii = valid ? i : (active ? td.y : 0);
    const int k = key_sorted[ii];
    const int cx = k % nc, cy = (k / nc) % nc, cz = k / (nc * nc);
    const double4_32a gi = pg[ii];
    const R4 pi = pr[ii];
    const T4 *ljrow = kLJ ? ljs + lj.tsort[ii] * lj.ntypes : nullptr;

    RowWalk wk;
    wk.w = w; wk.nc = nc; wk.part = part; wk.split = split;
    wk.cx = cx; wk.cy = cy; wk.cz = cz;
    // position of the target inside its own cell (for the ranges only); ranges are chosen a
    // little wider than r_c (a relative margin far above the rounding of the range
    // arithmetic), and the pair test decides with the exact cutoff
    wk.xl = (float)(gi.x - cx * side_d);
    wk.yl = (float)(gi.y - cy * side_d);
    wk.zl = (float)(gi.z - cz * side_d);
    wk.sidef = (float)side_d;
    wk.inv_side = (float)(1.0 / side_d);
    wk.rc2m = (float)rc2 * (1.0f + 1e-5f);
    wk.rn2m = kNear ? NK.rn2m : 0.0f;
    wk.valid = valid;
    wk.cell_start = cell_start;
    // x windows when the host chose them (use_xwin) and binning ordered every cell by x
    const bool xw = kFP32 && xwin && *unordered == 0;
    wk.rowctr = 0;
    wk.started = false;
    wk.in_row = false;
    wk.next_c0 = 0;

    // Staged walk over the rows of a RowWalk: item(sb, lo, hi, cur) for every staged item,
    // with [lo, hi) this target's part of the chunk in the buffer sb.  The two buffers and
    // their barrier phases carry over from one walk to the next.  False when a bounded wait
    // gave up.
    uint32_t phase[2] = {0u, 0u};
    int b = 0;
    auto next = [&](RowWalk &rw, RowItem &it) -> bool {
        return rw.template next<kCapR>(it, xw, (float)inv_s);
    };
    auto walk = [&](RowWalk &rw, auto &&item) -> bool {
        RowItem cur, nxt;
        bool have_cur = active && next(rw, cur);
        if (have_cur && lane == 0) {
            // (the buffer may have been read by the last walk, before its last __syncwarp)
            fence_proxy_async();
            issue_item(cur, pr, stage[warp][b], &bar[b]);
        }
        while (have_cur) {
            const bool have_nxt = next(rw, nxt);
            if (have_nxt && lane == 0) {
                // the other buffer was fully read before the last __syncwarp of the loop
                fence_proxy_async();
                issue_item(nxt, pr, stage[warp][b ^ 1], &bar[b ^ 1]);
            }
            if (!warp_wait(&bar[b], phase[b])) {
                // let a copy still in flight land before the warp leaves (bounded)
                if (have_nxt) warp_wait(&bar[b ^ 1], phase[b ^ 1]);
                return false;
            }
            phase[b] ^= 1u;
            const int lo = (cur.off0 > cur.c0 ? cur.off0 : cur.c0) - cur.c0;
            const int hi = (cur.off1 < cur.c0 + cur.cnt ? cur.off1 : cur.c0 + cur.cnt) - cur.c0;
            item(stage[warp][b], lo, hi, cur);
            __syncwarp();
            cur = nxt;
            have_cur = have_nxt;
            b ^= 1;
        }
        return true;
    };

    Acc acc{}, tot{}, comp{};     // sums of the current row, totals, Kahan compensation
    // Double-float near pairs (kNear): the near pairs (r < r_near) of every staged item are
    // queued in shared memory in the order they are found (candidate step, then lane) and
    // evaluated 32 at a time, one per lane; each target's results are added in queue order.
    NearTerm<kVir> nr;            // the Coulomb sums of this target (double-float), its virial
    int4 *qd = kNear ? nq_d[warp] : nullptr;
    int *qt = kNear ? nq_t[warp] : nullptr;
    int qn = 0;
    bool ok = walk(wk, [&](const R4 *sb, int lo, int hi, const RowItem &cur) {
        if constexpr (kFP32) {
            // the x window: along a target's range the candidates are in x order (cells in
            // order, each ordered by x), so their x displacements (int)(x_i - x_j) do not
            // increase, and with reach + side < L/2 the int32 differences are exact; two
            // binary searches of the staged records give the part inside [-xr, xr]
            if (cur.xr && lo < hi) {
                lo = first_within(sb, lo, hi, pi.x, cur.xr);
                hi = first_within(sb, lo, hi, pi.x, -cur.xr - 1);
            }
        }
        for (int j = lo + g; j < hi; j += G) {
            const R4 pj = sb[j];
            int tj = 0;
            if constexpr (kLJ) {
                const int q = cur.c0 + j;
                const int gidx = q < cur.u.lenA ? cur.u.sA + q
                               : (q < cur.u.lenA + cur.u.lenB ? cur.u.sB + (q - cur.u.lenA)
                                                              : cur.u.sC + (q - cur.u.lenA - cur.u.lenB));
                tj = lj.tsort[gidx];
            }
            if constexpr (kFP32) {
                pair_s<kDF, T4>(acc, (int)(pi.x - pj.x), (int)(pi.y - pj.y), (int)(pi.z - pj.z),
                                rec_q(pj), K, ljrow, tj);
            } else {
                // global coordinates, shifted by L where the row wraps
                const T yi = pi.y + (cy + cur.dy < 0 ? T(L_d) : (cy + cur.dy >= nc ? T(-L_d) : T(0)));
                const T zi = pi.z + (cz + cur.dz < 0 ? T(L_d) : (cz + cur.dz >= nc ? T(-L_d) : T(0)));
                const int q = cur.c0 + j;
                const T shift = q < cur.u.lenA ? T(L_d)
                              : (q >= cur.u.lenA + cur.u.lenB ? T(-L_d) : T(0));
                pair_d<T, T4>(acc, (pi.x + shift) - pj.x, yi - pj.y, zi - pj.z, (T)rec_q(pj), rc2,
                              beta, -beta * beta, two_b_rpi, ljrow, tj);
            }
        }
        acc_add_rows(tot, comp, acc);
        acc = Acc{};
        if constexpr (kNear) {
            const int nlo = (cur.noff0 > cur.c0 ? cur.noff0 : cur.c0) - cur.c0;
            const int nhi = (cur.noff1 < cur.c0 + cur.cnt ? cur.noff1 : cur.c0 + cur.cnt) - cur.c0;
            const int len = nhi > nlo ? nhi - nlo : 0;
            const int steps = __reduce_max_sync(0xffffffffu, len);
            for (int it = 0; it < steps; ++it) {
                bool hit = false;
                int4 e = make_int4(0, 0, 0, 0);
                if (it < len) {
                    const R4 pj = sb[nlo + it];
                    e = make_int4((int)(pi.x - pj.x), (int)(pi.y - pj.y), (int)(pi.z - pj.z),
                                  (int)pj.w);
                    const float r2f = r2_f32((float)e.x, (float)e.y, (float)e.z);
                    hit = r2f < K.rn2s && r2f > 0.0f;
                }
                const unsigned m = __ballot_sync(0xffffffffu, hit);
                if (hit) {
                    const int pos = qn + __popc(m & ((1u << lane) - 1u));
                    qd[pos] = e;
                    qt[pos] = lane;
                }
                qn += __popc(m);
                if (qn >= 32) {
                    __syncwarp();
                    near_flush<kVir>(nr, qd, qt, nq_l[warp], 32, lane, NK, ex2tab);
                    qn -= 32;
                    if (lane < qn) { qd[lane] = qd[32 + lane]; qt[lane] = qt[32 + lane]; }
                    __syncwarp();
                }
            }
        }
    });
    if constexpr (kFP32) {
        if (kNear && ok && qn > 0) {
            __syncwarp();
            near_flush<kVir>(nr, qd, qt, nq_l[warp], qn, lane, NK, ex2tab);
        }
        // the FP32 totals (less their Kahan compensation) join the near sums
        nr.fx = df_add(nr.fx, df_sum(tot.fx, -comp.fx));
        nr.fy = df_add(nr.fy, df_sum(tot.fy, -comp.fy));
        nr.fz = df_add(nr.fz, df_sum(tot.fz, -comp.fz));
        nr.phi = df_add(nr.phi, df_sum(tot.phi, -comp.phi));
        if constexpr (kVir) {
#pragma unroll
            for (int c = 0; c < 6; ++c) nr.w[c] += tot.w[c];
        }
    }
    if (!ok) {
        if (lane == 0) atomicOr(status, kStTimeout);
        if (split == 1) return;
    }
    acc = tot;
    // FP32: back from fixed-point units (forces 1 / S^2, potential, Coulomb virial and
    // Lennard-Jones force 1 / S), see pair_s
    const double fsc = kFP32 ? inv_s * inv_s : 1.0;
    const double psc = kFP32 ? inv_s : 1.0;
    // the Coulomb sums in FP64 (FP32: the FP32 totals and the near pairs, in double-float)
    double sx, sy, sz, sp;
    if constexpr (kFP32) {
        sx = (double)nr.fx.h + (double)nr.fx.l;
        sy = (double)nr.fy.h + (double)nr.fy.l;
        sz = (double)nr.fz.h + (double)nr.fz.l;
        sp = (double)nr.phi.h + (double)nr.phi.l;
        if constexpr (kVir) {
#pragma unroll
            for (int c = 0; c < 6; ++c) acc.w[c] = nr.w[c];
        }
    } else {
        sx = acc.fx; sy = acc.fy; sz = acc.fz; sp = acc.phi;
    }
    // combine the G lanes of every target (lanes t G .. t G + G - 1)
#pragma unroll
    for (int o = 1; o < G; o <<= 1) {
        acc_shfl_add(acc, o);
        sx += __shfl_xor_sync(0xffffffffu, sx, o);
        sy += __shfl_xor_sync(0xffffffffu, sy, o);
        sz += __shfl_xor_sync(0xffffffffu, sz, o);
        sp += __shfl_xor_sync(0xffffffffu, sp, o);
    }
    if (split > 1) {
        // every warp of the block reaches this barrier (none has returned with split > 1);
        // part 0 adds the other parts' sums in part order
        if (part > 0) {
            xacc[warp][lane] = acc;
            if constexpr (kFP32) xsum[warp][lane] = double4_32a{sx, sy, sz, sp};
        }
        __syncthreads();
        if (part > 0 || !active) return;
        for (int k = 1; k < split; ++k) {
            acc_add(acc, xacc[warp + k][lane]);
            if constexpr (kFP32) {
                const double4_32a o = xsum[warp + k][lane];
                sx += o.x; sy += o.y; sz += o.z; sp += o.w;
            }
        }
        if constexpr (!kFP32) { sx = acc.fx; sy = acc.fy; sz = acc.fz; sp = acc.phi; }
    }
    const double qi = (double)rec_q(pi);
    const bool mine = valid && g == 0;
    const double phi_i = psc * sp;
    if (mine) {
        double f[3] = {qi * fsc * sx, qi * fsc * sy, qi * fsc * sz};
        if constexpr (kLJ) {
            f[0] += psc * (double)acc.lj_f[0];
            f[1] += psc * (double)acc.lj_f[1];
            f[2] += psc * (double)acc.lj_f[2];
        }
        f_out[3 * (int64_t)i + 0] = f[0];
        f_out[3 * (int64_t)i + 1] = f[1];
        f_out[3 * (int64_t)i + 2] = f[2];
        phi_out[i] = phi_i;
    }
    const double e = warp_sum(mine ? qi * phi_i : 0.0);
    if (lane == 0) e_tile[grp] = e;
    acc_store_tile(acc, mine, qi, lane, vir_tile, vcap, lj.e_tile, grp, psc);
}

// All pairs with the minimum image (boxes too small for a cell stencil): one tile of 32
// targets per warp, every particle staged through the same double-buffered TMA path.  FP32:
// the fixed-point records (the difference of two fractions modulo 2^32 is the minimum-image
// displacement) and the pair arithmetic of the cell kernel (pair_s, FP32 near pairs with the
// exact r^2); FP64: the wrapped positions with an explicit minimum image.
template <class T, bool kVir, bool kLJ>
__global__ void __launch_bounds__(kWarps * 32)
k_real_allpairs(const typename Vec4<T>::type *__restrict__ pl, const uint4 *__restrict__ pu,
                int n, T L, T rc2, T beta, T two_b_rpi, ScaledK K, double inv_s,
                double *__restrict__ f_out, double *__restrict__ phi_out,
                double *__restrict__ e_tile, double *__restrict__ vir_tile, int64_t vcap,
                LJArgs lj, int *__restrict__ status)
{
    using T4 = typename Vec4<T>::type;
    constexpr bool kFP32 = sizeof(T) == 4;
    static_assert(sizeof(T4) == sizeof(uint4) || !kFP32, "FP32 records and float4 share a size");
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
    // (FP32: sigma^2 in units of S^2, S = inv_s^-1 the fixed-point step)
    if constexpr (kLJ) load_lj_table<T, T4>(ljs, lj, (double)rc2, kFP32 ? inv_s * inv_s : 1.0);
    const int tile = blockIdx.x * kWarps + warp;
    if (tile * 32 >= n) return;
    const int i = tile * 32 + lane;
    const bool valid = i < n;
    const int ii = valid ? i : n - 1;
    // the staged records: FP32 the fixed-point fractions, FP64 the wrapped positions
    const T4 *src = kFP32 ? reinterpret_cast<const T4 *>(pu) : pl;
    const T4 pi = src[ii];
    const uint4 pi_u = kFP32 ? pu[ii] : make_uint4(0, 0, 0, 0);
    const T4 *ljrow = kLJ ? ljs + lj.tsort[ii] * lj.ntypes : nullptr;
    const T invL = T(1) / L;
    using Acc = PairAcc<T, kVir, kLJ>;
    Acc acc{}, tot{}, comp{};     // sums of the current chunk, totals, Kahan compensation
    const T nb2 = kFP32 ? -beta * beta * T(kLog2e) : -beta * beta;
    uint32_t phase[2] = {0u, 0u};
    const int nchunks = (n + kCapAll - 1) / kCapAll;
    if (lane == 0) {
        int cnt = min(kCapAll, n);
        mbar_expect_tx(&bar[0], cnt * (uint32_t)sizeof(T4));
        tma_bulk_g2s(buf[0], src, cnt * (uint32_t)sizeof(T4), &bar[0]);
    }
    bool ok = true;
    int b = 0;
    for (int c = 0; c < nchunks; ++c) {
        if (c + 1 < nchunks && lane == 0) {
            int g = (c + 1) * kCapAll, cnt = min(kCapAll, n - g);
            fence_proxy_async();
            mbar_expect_tx(&bar[b ^ 1], cnt * (uint32_t)sizeof(T4));
            tma_bulk_g2s(buf[b ^ 1], src + g, cnt * (uint32_t)sizeof(T4), &bar[b ^ 1]);
        }
        if (!warp_wait(&bar[b], phase[b])) { ok = false; break; }
        phase[b] ^= 1u;
        const int cnt = min(kCapAll, n - c * kCapAll);
        const T4 *sb = buf[b];
        for (int j = 0; j < cnt; ++j) {
            const int tj = kLJ ? lj.tsort[c * kCapAll + j] : 0;
            if constexpr (kFP32) {
                const uint4 pj = reinterpret_cast<const uint4 *>(sb)[j];
                pair_s<false, T4>(acc, (int)(pi_u.x - pj.x), (int)(pi_u.y - pj.y),
                                  (int)(pi_u.z - pj.z), __uint_as_float(pj.w), K, ljrow, tj);
            } else {
                T4 p = sb[j];
                T dx = pi.x - p.x, dy = pi.y - p.y, dz = pi.z - p.z;
                dx -= L * rint(dx * invL);
                dy -= L * rint(dy * invL);
                dz -= L * rint(dz * invL);
                // evaluate the pair at the minimum image: shift the partner, keep the target
                T4 pj = p;
                pj.x = pi.x - dx; pj.y = pi.y - dy; pj.z = pi.z - dz;
                pair<T, T4>(acc, pj, pi.x, pi.y, pi.z, rc2, beta, nb2, two_b_rpi, ljrow, tj);
            }
        }
        acc_add_rows(tot, comp, acc);
        acc = Acc{};
        __syncwarp();
        b ^= 1;
    }
    if (!ok) {
        if (lane == 0) atomicOr(status, kStTimeout);
        warp_wait(&bar[b ^ 1], phase[b ^ 1]);
        return;
    }
    // FP32: back from fixed-point units (forces 1 / S^2, potential, Coulomb virial and
    // Lennard-Jones force 1 / S), see pair_s
    const double fsc = kFP32 ? inv_s * inv_s : 1.0;
    const double psc = kFP32 ? inv_s : 1.0;
    const double qi = kFP32 ? (double)__uint_as_float(pi_u.w) : (double)pi.w;
    const double sx = (double)tot.fx - (double)comp.fx, sy = (double)tot.fy - (double)comp.fy,
                 sz = (double)tot.fz - (double)comp.fz, sp = (double)tot.phi - (double)comp.phi;
    const double phi_i = psc * sp;
    if (valid) {
        double f[3] = {qi * fsc * sx, qi * fsc * sy, qi * fsc * sz};
        if constexpr (kLJ) {
            f[0] += psc * (double)tot.lj_f[0];
            f[1] += psc * (double)tot.lj_f[1];
            f[2] += psc * (double)tot.lj_f[2];
        }
        f_out[3 * (int64_t)i + 0] = f[0];
        f_out[3 * (int64_t)i + 1] = f[1];
        f_out[3 * (int64_t)i + 2] = f[2];
        phi_out[i] = phi_i;
    }
    const double e = warp_sum(valid ? qi * phi_i : 0.0);
    if (lane == 0) e_tile[tile] = e;
    acc_store_tile(tot, valid, qi, lane, vir_tile, vcap, lj.e_tile, tile, psc);
}

// Warps per group of targets of the cell kernel: 4 below 24 groups per SM, 2 below 32, else
// 1 (measured on GB300, steps in ms with 1 / 2 / 4 warps per group: 32,768 ions 0.52 / 0.47 /
// 0.43; 65,536: 1.10 / 1.05 / 1.03; 131,072: 2.87 / 2.92 / 2.96; 262,144: 4.34 / 4.33 / 4.40).
int real_split(int64_t groups, int num_sms)
{
    if (groups < 24 * (int64_t)num_sms) return 4;
    return groups < 32 * (int64_t)num_sms ? 2 : 1;
}

template <class T, bool kVir, bool kLJ>
cudaError_t launch_real_t(Plan &p, int64_t n, const typename Vec4<T>::type *pl, cudaStream_t st)
{
    Workspace &ws = p.ws;
    double *vir = kVir ? ws.vir_tile : nullptr;
    const int64_t vcap = real_tile_capacity(p, n);
    LJArgs lj{ws.type_sorted, p.lj_tab_d, p.lj_ntypes, ws.elj_tile};
    const size_t smem = (size_t)kWarps * 2 * kCapAll * sizeof(typename Vec4<T>::type);
    const T beta = (T)p.beta, rc2 = (T)(p.rc * p.rc);
    const T tbr = (T)(2.0 * p.beta / sqrt(kPi));
    // FP32: constants in units of the fixed-point step S = L / 2^32 (see pair_s); near pairs
    // are those within 2.5 mean particle spacings (at most r_c)
    const double S = p.L / 4294967296.0;
    const double spacing = cbrt(p.L * p.L * p.L / (double)(n > 0 ? n : 1));
    const double rnear = fmin(2.5 * spacing, p.rc);
    ScaledK K;
    K.rc2s = (float)(p.rc * p.rc / (S * S));
    K.rn2s = (float)(rnear * rnear / (S * S));
    K.beta_s = (float)(p.beta * S);
    K.nb2l_s = (float)(-p.beta * p.beta * S * S * 1.4426950408889634);
    K.c_s = (float)(2.0 * p.beta / sqrt(kPi) * S);
    K.cb2_s = (float)(2.0 * p.beta / sqrt(kPi) * S * (p.beta * S) * (p.beta * S));
    cudaError_t e;
    if (p.w == 0) {
        auto kern = k_real_allpairs<T, kVir, kLJ>;
        e = smem_optin((const void *)kern);
        if (e != cudaSuccess) return e;
        int tiles = (int)((n + 31) / 32);
        kern<<<(tiles + kWarps - 1) / kWarps, kWarps * 32, smem, st>>>(
            pl, ws.pu, (int)n, (T)p.L, rc2, beta, tbr, K, 1.0 / S, ws.f_real, ws.phi_real,
            ws.e_tile, vir, vcap, lj, p.d_status);
    } else {
        // (the FP64 kernel has no near-pair modes: one instantiation)
        auto kern = (sizeof(T) == 4 && p.near_df) ? k_real_rows<T, 1, kVir, kLJ, sizeof(T) == 4>
                                                  : k_real_rows<T, 1, kVir, kLJ, false>;
        const int64_t groups = real_tile_capacity(p, n);
        // two or four warps per group of targets when one warp per group would leave the SMs
        // short of warps
        const int split = real_split(groups, p.num_sms);
        const typename RowRec<T>::type *pr;
        if constexpr (sizeof(T) == 4) pr = ws.pu;
        else pr = ws.pg;
        // double-float constants of the near pairs, and their reach (with the range margin)
        NearK NK;
        const double bs = p.beta * S, cs = 2.0 * p.beta / sqrt(kPi) * S;
        NK.beta_h = (float)bs;
        NK.beta_l = (float)(bs - (double)NK.beta_h);
        NK.c_h = (float)cs;
        NK.c_l = (float)(cs - (double)NK.c_h);
        NK.rn2m = (float)(rnear * rnear) * (1.0f + 1e-5f);
        const int xwin = sizeof(T) == 4 && use_xwin(p);
        kern<<<(unsigned)((groups * split + kWarps - 1) / kWarps), kWarps * 32, 0, st>>>(
            pr, ws.pg, ws.key_sorted, ws.cell_start, ws.tiles, ws.tile_off + p.nc * p.nc,
            (int)n, p.nc, p.w, p.cell_side, p.L, rc2, beta, tbr, K, NK, 1.0 / S, split, xwin,
            ws.unordered, ws.f_real, ws.phi_real, ws.e_tile, vir, vcap, lj, p.d_status);
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
    // tiles never leave a row: at most one ragged tile per row
    return n / real_tile_size(p) + (int64_t)p.nc * p.nc + 1;
}

// targets per warp: 32 in all-pairs mode, else 32 / G with G lanes per target
int real_tile_size(const Plan &p) { return p.w == 0 ? 32 : 32 / p.real_tile; }

// Lanes per target of the cell kernel: one, so that the 32 targets of a warp share every
// staged row (measured on GB300, real-space kernel alone, ms with 1 / 2 / 4 lanes per target:
// 32,768 ions 0.152 / 0.168 / 0.202; 262,144: 1.42 / 1.63 / 2.15; 2,097,152: 22.2 / 24.6 /
// 28.8).  The kernel is templated on the lane count; this build instantiates one lane.
int real_tile_for(int, double)
{
    return 1;
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
