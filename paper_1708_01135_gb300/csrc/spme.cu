// Smooth particle-mesh Ewald (SPME): the reciprocal part on a K^3 mesh, the successor that
// the paper names for large N (Sections 1 and 5).  The method is that of Essmann et al.,
// J. Chem. Phys. 103, 8577 (1995), in the paper's Gaussian units:
//
//   u_a = K x_a / L (scaled fractional coordinates), M_p the cardinal B-spline of even order
//   p, Q(k) = sum_i q_i prod_a M_p(u_ia - k_a) (periodically wrapped),
//   E_recip = 1/2 sum_{m != 0} G(m) |F(Q)(m)|^2,
//   G(m) = exp(-pi^2 |m~|^2 / beta^2) / (pi V |m~|^2) prod_a |b(m_a)|^2,  m~ = m / L,
//   |b(m)|^2 = 1 / |sum_{k=0}^{p-2} M_p(k+1) exp(2 pi i m k / K)|^2,
//   phi_mesh = F^-1[G F(Q)] (unnormalised inverse), F_i = -q_i (K/L) sum_k grad M phi_mesh,
//   phi_i = sum_k M phi_mesh (so that E = 1/2 sum q_i phi_i).
//
// GPU design:
//   * spread: one block per brick of cells of the real-space cell grid (the particles are
//     sorted by cell) spreads the brick's charges into a tile of the mesh held in shared
//     memory, with no atomics: warp w of the p warps owns the tile planes x = w (mod p), so
//     every tile point is updated by one warp, particle after particle in slot order.  The
//     tile is then added to a fixed-point mesh (2^-36 resolution) with one 64-bit integer
//     atomic per nonzero point.  Integer addition is associative, so the mesh, and
//     everything after it, is bit-identical from run to run whatever order the bricks
//     finish in.  (A grid too coarse for tiles falls back to one thread per particle with
//     p^3 atomics, e.g. a single cell on a small box);
//   * convert (fixed point -> FP64/FP32, and re-zero the fixed-point mesh for the next call),
//     cuFFT real-to-complex transform (a plain library FFT);
//   * influence: G is the product of three per-axis tables and 1 / |m~|^2, computed on the
//     fly (no K^3 coefficient array, FP32 arithmetic on the FP32 mesh); the same pass forms
//     the energy and virial partials (fixed-order sums, FP64 across groups of 16 entries)
//     and scales the spectrum by G;
//   * cuFFT complex-to-real transform, then gather: per brick, the tile of the potential
//     mesh is copied to shared memory, and one thread per particle sums over its p^3 points
//     and writes its own force and potential (no atomics).
// The mixed and FP32 plans use FP32 splines, mesh and FFT; the FP64 plan FP64 throughout.
#include <cuda_runtime.h>
#include <cufft.h>
#include <math.h>
#include <stdint.h>

#include <new>
#include <type_traits>
#include <vector>

#include "ewald_internal.cuh"

namespace ew {

struct SpmeState {
    int K = 0, order = 0;
    bool fp32 = false;
    cufftHandle fwd = 0, inv = 0;
    bool have_fwd = false, have_inv = false;
    unsigned long long *qfix = nullptr;   // [K^3] fixed-point charge mesh
    void *mesh = nullptr;                 // [K^3] real mesh (charges, then potentials)
    void *spec = nullptr;                 // [K][K][K/2 + 1] complex spectrum
    double2 *axis = nullptr;              // [K]: (|b(m)|^2 exp(-pi^2 s^2 / (beta L)^2), s / L)
    double *part = nullptr;               // [7][nblk] energy and virial partials
    int nblk = 0;                         // blocks of the spectrum pass
    double axis_beta = 0, axis_L = 0;     // parameters the axis table was built for
    // brick tiling of the spreading for the plan's current cell grid (tile_nc = -1: not
    // chosen yet; bc = 0: no tile fits, spread particle by particle)
    int tile_nc = -1, bc = 0, nbk = 0, W = 0, S = 24, chunk = 0;
    size_t smem = 0;                      // dynamic shared memory of the spreading blocks
    // the gather's bricks (larger: one thread per particle wants >= 128 particles a block)
    int bc_g = 0, nbk_g = 0, W_g = 0;
    int64_t tile_n = -1;                  // particle count the gather's bricks were chosen for
    size_t smem_g = 0;
};

namespace {

constexpr double kFixScale = 68719476736.0;          // 2^36
constexpr double kFixInv = 1.0 / 68719476736.0;
constexpr int kThreads = 256;

// M_P(w + j) for j = 0..P-1 (w in [0, 1)) by the order recursion
// M_n(t) = t/(n-1) M_{n-1}(t) + (n-t)/(n-1) M_{n-1}(t-1), from M_2(w) = w, M_2(w + 1) = 1 - w;
// with D, also dM_P/du(w + j) = M_{P-1}(w + j) - M_{P-1}(w + j - 1).
template <class T, int P, bool D>
__device__ __forceinline__ void spline(T w, T (&c)[P], T (&d)[P])
{
#pragma unroll
    for (int j = 0; j < P; ++j) c[j] = T(0);
    c[0] = w;
    c[1] = T(1) - w;
#pragma unroll
    for (int n = 3; n <= P; ++n) {
        if (D && n == P) {
            d[0] = c[0];
#pragma unroll
            for (int j = 1; j < P; ++j) d[j] = c[j] - c[j - 1];
        }
        const T inv = T(1) / T(n - 1);
#pragma unroll
        for (int j = n - 1; j >= 1; --j) c[j] = ((w + T(j)) * c[j] + (T(n) - w - T(j)) * c[j - 1]) * inv;
        c[0] = w * c[0] * inv;
    }
}

// Mesh indices of the P points of one axis: base - j (mod K), and the weight argument w.
__device__ __forceinline__ void axis_pos(double x, double kl, int K, int &base, double &w)
{
    const double u = x * kl;            // x in [0, L): u in [0, K]
    const double f = floor(u);
    w = u - f;
    base = (int)f;
    if (base >= K) base -= K;
}

// One particle's P^3 charge weights, added to the fixed-point mesh with integer atomics.
template <class T, int P>
__device__ void spread_one(const double4_32a &r, int K, double kl,
                           unsigned long long *__restrict__ qfix)
{
    int b[3];
    double w[3];
    axis_pos(r.x, kl, K, b[0], w[0]);
    axis_pos(r.y, kl, K, b[1], w[1]);
    axis_pos(r.z, kl, K, b[2], w[2]);
    T cx[P], cy[P], cz[P], dd[P];
    spline<T, P, false>((T)w[0], cx, dd);
    spline<T, P, false>((T)w[1], cy, dd);
    spline<T, P, false>((T)w[2], cz, dd);
    const T q = (T)r.w;
    int iz[P];
#pragma unroll
    for (int c = 0; c < P; ++c) iz[c] = b[2] - c < 0 ? b[2] - c + K : b[2] - c;
#pragma unroll 1
    for (int a = 0; a < P; ++a) {
        const int ix = b[0] - a < 0 ? b[0] - a + K : b[0] - a;
        const T qa = q * cx[a];
#pragma unroll 1
        for (int bb = 0; bb < P; ++bb) {
            const int iy = b[1] - bb < 0 ? b[1] - bb + K : b[1] - bb;
            const T qab = qa * cy[bb];
            unsigned long long *row = qfix + ((int64_t)ix * K + iy) * K;
#pragma unroll
            for (int c = 0; c < P; ++c) {
                const long long v = llrint((double)(qab * cz[c]) * kFixScale);
                atomicAdd(row + iz[c], (unsigned long long)v);
            }
        }
    }
}

// Spreading particle by particle (grids with no room for tiles).
template <class T, int P>
__global__ void __launch_bounds__(kThreads)
k_spme_spread(int64_t n, const double4_32a *__restrict__ pg, int K, double kl,
              unsigned long long *__restrict__ qfix)
{
    const int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x;
    if (i >= n) return;
    spread_one<T, P>(pg[i], K, kl, qfix);
}

// Mesh index o + l wrapped into [0, K), for o + l in [-K, 2K).
__device__ __forceinline__ int wrap_mesh(int g, int K)
{
    return g < 0 ? g + K : (g >= K ? g - K : g);
}

// The fixed-point value of a tile sum (2^-36 resolution, round to nearest even), equal to
// llrint(v * 2^36) in either precision.  For FP32 it is put together from 32-bit conversions
// (a 64-bit conversion runs on the FP64 units): with s = 16 |v| and h = floor(s),
// |v| 2^36 = h 2^32 + r, r = (s - h) 2^32 in [0, 2^32), where s, h, the fraction s - h
// (s >= 0) and r are exact in FP32 (r is a float below 2^32, so it rounds to at most
// 2^32 - 256), and h 2^32 is an even integer, so rounding r rounds |v| 2^36 (ties to even
// included); rounding to nearest even is odd-symmetric, so the sign is applied last.
// |v| < 2^26 keeps h in int range.
__device__ __forceinline__ long long to_fix(float v)
{
    const float s = fabsf(v) * 16.0f;
    const float h = floorf(s);
    const float r = (s - h) * 4294967296.0f;
    const long long m = (long long)(int)h * 4294967296ll + (long long)__float2uint_rn(r);
    return v < 0.0f ? -m : m;
}
__device__ __forceinline__ long long to_fix(double v) { return __double2ll_rn(v * kFixScale); }

// Tiled spreading (see the file comment).  Block b is the brick (bx, by, bz) of bc^3 cells;
// its particles are the slot ranges of its cell rows.  The tile covers mesh points
// [o, o + W) per axis with o = floor(c0 K / nc) - P: every particle of cells [c0, c1) has
// its mesh base floor(u) in [o + P, floor(c1 K / nc)], up to rounding, and W leaves one
// point of margin at each end; a particle found outside all the same is spread directly
// into the global mesh.  The tile is stored [W][W][S] (S >= W a compile-time row pitch, so
// that offsets inside one plane of a particle's footprint are constants; S = 24 or 40 keeps
// the P x P points a warp updates in distinct shared-memory banks for P = 8).  After the tile, per
// particle of the current chunk: its 3 x P weights (the x weights times its charge), then
// its tile offset and its x base modulo P.
template <class T, int P, int S>
__global__ void __launch_bounds__(P * 32)
k_spme_spread_tile(const double4_32a *__restrict__ pg, const int *__restrict__ cell_start,
                   int nc, int bc, int nbk, int W, int chunk, int K, double kl,
                   unsigned long long *__restrict__ qfix)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    __shared__ int rfirst[64], rpre[65];
    const int S2 = W * S;          // plane stride
    const int TV = W * S2;
    T *tile = reinterpret_cast<T *>(smraw);
    T *wts = tile + TV;
    int2 *info = reinterpret_cast<int2 *>(
        smraw + (((TV + (size_t)chunk * 3 * P) * sizeof(T) + 7) & ~(size_t)7));
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    constexpr int nth = P * 32;
    constexpr int NI = (P * P + 31) / 32;
    const int b = blockIdx.x;
    const int bx = b % nbk, by = (b / nbk) % nbk, bz = b / (nbk * nbk);
    const int cx0 = bx * bc, cy0 = by * bc, cz0 = bz * bc;
    const int cx1 = min(nc, cx0 + bc), cy1 = min(nc, cy0 + bc), cz1 = min(nc, cz0 + bc);
    const int o[3] = {(int)(((int64_t)cx0 * K) / nc) - P, (int)(((int64_t)cy0 * K) / nc) - P,
                      (int)(((int64_t)cz0 * K) / nc) - P};
    const int nry = cy1 - cy0, nr = nry * (cz1 - cz0);
    if (tid < nr) {
        const int base = ((cz0 + tid / nry) * nc + cy0 + tid % nry) * nc;
        const int f = cell_start[base + cx0];
        rfirst[tid] = f;
        rpre[tid + 1] = cell_start[base + cx1] - f;
    }
    for (int t = tid; t < TV; t += nth) tile[t] = T(0);
    // this lane's points (b, c) of a particle's P x P footprint in one plane: offsets from
    // the particle's base point and the positions of their weights
    int off[NI], wy_i[NI], wz_i[NI];
    bool has[NI];
#pragma unroll
    for (int i = 0; i < NI; ++i) {
        const int idx = lane + 32 * i;
        has[i] = idx < P * P;
        const int bb = has[i] ? idx / P : 0, cc = has[i] ? idx % P : 0;
        off[i] = -bb * S - cc;
        wy_i[i] = P + bb;
        wz_i[i] = 2 * P + cc;
    }
    __syncthreads();
    if (tid == 0) {
        rpre[0] = 0;
        for (int r = 0; r < nr; ++r) rpre[r + 1] += rpre[r];
    }
    __syncthreads();
    const int total = rpre[nr];
    int r = 0;
    for (int c0 = 0; c0 < total; c0 += chunk) {
        const int cnt = min(chunk, total - c0);
        if (tid < cnt) {
            const int f = c0 + tid;
            while (rpre[r + 1] <= f) ++r;
            const double4_32a pr = pg[rfirst[r] + (f - rpre[r])];
            const double u[3] = {pr.x * kl, pr.y * kl, pr.z * kl};
            int l[3];
            T w[3];
            bool inside = true;
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                const double fl = floor(u[a]);
                l[a] = (int)fl - o[a];
                w[a] = (T)(u[a] - fl);
                inside = inside && l[a] >= P - 1 && l[a] < W;
            }
            T *wp = wts + (size_t)tid * 3 * P;
            if (inside) {
                T c[P], d[P];
                const T q = (T)pr.w;
                spline<T, P, false>(w[0], c, d);
#pragma unroll
                for (int j = 0; j < P; ++j) wp[j] = q * c[j];
#pragma unroll
                for (int a = 1; a < 3; ++a) {
                    spline<T, P, false>(w[a], c, d);
#pragma unroll
                    for (int j = 0; j < P; ++j) wp[a * P + j] = c[j];
                }
                info[tid] = make_int2(l[0] * S2 + l[1] * S + l[2], l[0] % P);
            } else {
                spread_one<T, P>(pr, K, kl, qfix);
#pragma unroll
                for (int j = 0; j < 3 * P; ++j) wp[j] = T(0);
                info[tid] = make_int2((P - 1) * (S2 + S + 1), P - 1);
            }
        }
        __syncthreads();
        for (int j = 0; j < cnt; ++j) {
            const int2 in = info[j];
            int a = in.y - warp;
            if (a < 0) a += P;
            const T *wp = wts + (size_t)j * 3 * P;
            const T qa = wp[a];
            T *pt = tile + (in.x - a * S2);
#pragma unroll
            for (int i = 0; i < NI; ++i)
                if (has[i]) pt[off[i]] += qa * wp[wy_i[i]] * wp[wz_i[i]];
            __syncwarp();
        }
        __syncthreads();
    }
    // the tile into the global mesh: warps step over the rows (x, y), lanes along z
    for (int lx = 0; lx < W; ++lx) {
        const int gx = wrap_mesh(o[0] + lx, K);
        for (int ly = warp; ly < W; ly += P) {
            unsigned long long *dst = qfix + ((int64_t)gx * K + wrap_mesh(o[1] + ly, K)) * K;
            const T *src = tile + lx * S2 + ly * S;
            for (int lz = lane; lz < W; lz += 32) {
                const T v = src[lz];
                if (v != T(0))
                    atomicAdd(dst + wrap_mesh(o[2] + lz, K), (unsigned long long)to_fix(v));
            }
        }
    }
}

template <class T>
__global__ void k_spme_convert(int64_t m, unsigned long long *__restrict__ qfix, T *__restrict__ mesh)
{
    const int64_t t = (int64_t)blockIdx.x * kThreads + threadIdx.x;
    if (t >= m) return;
    mesh[t] = (T)((double)(long long)qfix[t] * kFixInv);
    qfix[t] = 0ull;
}

// Spectrum pass over the K x K x (K/2 + 1) half spectrum: energy and virial partials of
// 1/2 sum_m G |F(Q)|^2 (entries m_z = 0 and m_z = K/2 stand for themselves, the others also
// for their conjugate partners) and spec <- G spec.  Arithmetic in the mesh type T; each
// thread adds its terms in T over groups of 16 entries and the group sums in FP64.  Block b
// takes the entries b * 256 + t + j * (gridDim.x * 256) in order, then a fixed tree; part
// holds [7][gridDim.x] block sums (energy, then the virial xx yy zz xy xz yz).
template <class T, class T2>
__global__ void __launch_bounds__(kThreads)
k_spme_influence(int K, const double2 *__restrict__ axis, double inv_piV, double pi2_b2,
                 T2 *__restrict__ spec, double *__restrict__ part)
{
    __shared__ double red[7][kThreads];
    const int Kh = K / 2 + 1;
    const int64_t tot = (int64_t)K * K * Kh;
    const int t = threadIdx.x;
    double acc[7] = {0, 0, 0, 0, 0, 0, 0};
    T grp[7] = {0, 0, 0, 0, 0, 0, 0};
    int ng = 0;
    const T ipv = (T)inv_piV, pb = (T)pi2_b2;
    for (int64_t e = (int64_t)blockIdx.x * kThreads + t; e < tot; e += (int64_t)gridDim.x * kThreads) {
        const int mz = (int)(e % Kh);
        const int64_t r = e / Kh;
        const int my = (int)(r % K), mx = (int)(r / K);
        const double2 ax = axis[mx], ay = axis[my], az = axis[mz];
        const T sx = (T)ax.y, sy = (T)ay.y, sz = (T)az.y;
        const T m2 = sx * sx + sy * sy + sz * sz;
        T2 v = spec[e];
        if (e != 0) {
            const T G = (T)ax.x * (T)ay.x * (T)az.x * ipv / m2;
            const T a = G * (v.x * v.x + v.y * v.y);
            const bool single = mz == 0 || 2 * mz == K;    // stands for itself only
            const T hw = single ? T(0.5) * a : a;           // 1/2 x (1 or 2)
            const T c = T(2) * (T(1) / m2 + pb);
            // an entry that also stands for its conjugate partner (-m): the partner's signed
            // frequencies are -s, except on a Nyquist index K/2, which is +K/2 for both
            // (the mesh cannot tell +K/2 from -K/2), so there the off-diagonal products of
            // the pair cancel
            const bool nx = 2 * mx == K, ny = 2 * my == K;
            const T fxy = (!single && nx != ny) ? T(0) : T(1);
            const T fxz = (!single && nx) ? T(0) : T(1), fyz = (!single && ny) ? T(0) : T(1);
            grp[0] += hw;
            grp[1] += hw * (T(1) - c * sx * sx);
            grp[2] += hw * (T(1) - c * sy * sy);
            grp[3] += hw * (T(1) - c * sz * sz);
            grp[4] -= fxy * hw * c * sx * sy;
            grp[5] -= fxz * hw * c * sx * sz;
            grp[6] -= fyz * hw * c * sy * sz;
            v.x *= G;
            v.y *= G;
        } else {
            v.x = 0;
            v.y = 0;
        }
        spec[e] = v;
        if (++ng == 16) {
#pragma unroll
            for (int c = 0; c < 7; ++c) { acc[c] += (double)grp[c]; grp[c] = T(0); }
            ng = 0;
        }
    }
#pragma unroll
    for (int c = 0; c < 7; ++c) red[c][t] = acc[c] + (double)grp[c];
    __syncthreads();
    for (int o = kThreads / 2; o > 0; o >>= 1) {
        if (t < o) {
#pragma unroll
            for (int c = 0; c < 7; ++c) red[c][t] += red[c][t + o];
        }
        __syncthreads();
    }
    if (t < 7) part[t * gridDim.x + blockIdx.x] = red[t][0];
}

// Shift the weights of one axis down by one (after plane a, entry 0 holds plane a + 1's):
// keeps the plane loop rolled without indexing register arrays by the loop counter.
template <class T, int P>
__device__ __forceinline__ void shift_down(T (&c)[P], T (&d)[P])
{
#pragma unroll
    for (int j = 0; j + 1 < P; ++j) { c[j] = c[j + 1]; d[j] = d[j + 1]; }
}

// One particle from the global mesh (periodic indices; grids with no room for tiles and
// particles outside their tile).
template <class T, int P>
__device__ void gather_one(const double4_32a &r, int K, double kl, const T *__restrict__ mesh,
                           double *__restrict__ f, double *__restrict__ phi)
{
    int b[3];
    double w[3];
    axis_pos(r.x, kl, K, b[0], w[0]);
    axis_pos(r.y, kl, K, b[1], w[1]);
    axis_pos(r.z, kl, K, b[2], w[2]);
    T cx[P], cy[P], cz[P], dx[P], dy[P], dz[P];
    spline<T, P, true>((T)w[0], cx, dx);
    spline<T, P, true>((T)w[1], cy, dy);
    spline<T, P, true>((T)w[2], cz, dz);
    int iz[P], iy[P];
#pragma unroll
    for (int c = 0; c < P; ++c) {
        iz[c] = b[2] - c < 0 ? b[2] - c + K : b[2] - c;
        iy[c] = (b[1] - c < 0 ? b[1] - c + K : b[1] - c) * K;
    }
    T s = T(0), gx = T(0), gy = T(0), gz = T(0);
#pragma unroll 1
    for (int a = 0; a < P; ++a) {
        const int ix = b[0] - a < 0 ? b[0] - a + K : b[0] - a;
        const T *pl = mesh + (int64_t)ix * K * K;
        T sa = T(0), ga = T(0), gza = T(0);
#pragma unroll
        for (int bb = 0; bb < P; ++bb) {
            const T *row = pl + iy[bb];
            T sz = T(0), dzs = T(0);
#pragma unroll
            for (int c = 0; c < P; ++c) {
                const T v = row[iz[c]];
                sz += cz[c] * v;
                dzs += dz[c] * v;
            }
            sa += cy[bb] * sz;
            ga += dy[bb] * sz;
            gza += cy[bb] * dzs;
        }
        s += cx[0] * sa;
        gx += dx[0] * sa;
        gy += cx[0] * ga;
        gz += cx[0] * gza;
        shift_down<T, P>(cx, dx);
    }
    const double qk = -(double)r.w * kl;
    f[0] = qk * (double)gx;
    f[1] = qk * (double)gy;
    f[2] = qk * (double)gz;
    *phi = (double)s;
}

// Gather particle by particle from the global mesh (grids with no room for tiles).
template <class T, int P>
__global__ void __launch_bounds__(kThreads)
k_spme_gather(int64_t n, const double4_32a *__restrict__ pg, int K, double kl,
              const T *__restrict__ mesh, double *__restrict__ f, double *__restrict__ phi)
{
    const int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x;
    if (i >= n) return;
    gather_one<T, P>(pg[i], K, kl, mesh, f + 3 * i, phi + i);
}

// Tiled gather: bricks of cells as for the spreading (larger ones: one thread per particle
// wants >= 128 particles a block).  The block first copies the W^3 tile of the potential
// mesh that its particles reach into shared memory (rows along z, coalesced), then every
// thread takes particles of the brick and sums over the tile, one plane of the footprint at
// a time (row offsets inside a plane are multiples of W, points along a row constants).  A
// particle found outside the tile reads the global mesh instead.
template <class T, int P>
__global__ void __launch_bounds__(kThreads)
k_spme_gather_tile(const double4_32a *__restrict__ pg, const int *__restrict__ cell_start,
                   int nc, int bc, int nbk, int W, int K, double kl, const T *__restrict__ mesh,
                   double *__restrict__ f, double *__restrict__ phi)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    __shared__ int rfirst[64], rpre[65];
    const int W2 = W * W;
    T *tile = reinterpret_cast<T *>(smraw);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    constexpr int nw = kThreads / 32;
    const int b = blockIdx.x;
    const int bx = b % nbk, by = (b / nbk) % nbk, bz = b / (nbk * nbk);
    const int cx0 = bx * bc, cy0 = by * bc, cz0 = bz * bc;
    const int cx1 = min(nc, cx0 + bc), cy1 = min(nc, cy0 + bc), cz1 = min(nc, cz0 + bc);
    const int o[3] = {(int)(((int64_t)cx0 * K) / nc) - P, (int)(((int64_t)cy0 * K) / nc) - P,
                      (int)(((int64_t)cz0 * K) / nc) - P};
    const int nry = cy1 - cy0, nr = nry * (cz1 - cz0);
    if (tid < nr) {
        const int base = ((cz0 + tid / nry) * nc + cy0 + tid % nry) * nc;
        const int f0 = cell_start[base + cx0];
        rfirst[tid] = f0;
        rpre[tid + 1] = cell_start[base + cx1] - f0;
    }
    // asynchronous element copies (cp.async): every load of the tile is in flight at once
    for (int lx = 0; lx < W; ++lx) {
        const T *pl = mesh + (int64_t)wrap_mesh(o[0] + lx, K) * K * K;
        for (int ly = warp; ly < W; ly += nw) {
            const T *src = pl + (int64_t)wrap_mesh(o[1] + ly, K) * K;
            T *dst = tile + lx * W2 + ly * W;
            for (int lz = lane; lz < W; lz += 32)
                asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(
                                 (uint32_t)__cvta_generic_to_shared(dst + lz)),
                             "l"(src + wrap_mesh(o[2] + lz, K)), "n"((int)sizeof(T))
                             : "memory");
        }
    }
    asm volatile("cp.async.wait_all;" ::: "memory");
    __syncthreads();
    if (tid == 0) {
        rpre[0] = 0;
        for (int r = 0; r < nr; ++r) rpre[r + 1] += rpre[r];
    }
    __syncthreads();
    const int total = rpre[nr];
    int r = 0;
    for (int fi = tid; fi < total; fi += kThreads) {
        while (rpre[r + 1] <= fi) ++r;
        const int slot = rfirst[r] + (fi - rpre[r]);
        const double4_32a pr = pg[slot];
        const double u[3] = {pr.x * kl, pr.y * kl, pr.z * kl};
        int l[3];
        T w[3];
        bool inside = true;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const double fl = floor(u[a]);
            l[a] = (int)fl - o[a];
            w[a] = (T)(u[a] - fl);
            inside = inside && l[a] >= P - 1 && l[a] < W;
        }
        if (!inside) {
            gather_one<T, P>(pr, K, kl, mesh, f + 3 * (int64_t)slot, phi + slot);
            continue;
        }
        T cx[P], cy[P], cz[P], dx[P], dy[P], dz[P];
        spline<T, P, true>(w[0], cx, dx);
        spline<T, P, true>(w[1], cy, dy);
        spline<T, P, true>(w[2], cz, dz);
        const T *base = tile + l[0] * W2 + l[1] * W + l[2];
        T s = T(0), gx = T(0), gy = T(0), gz = T(0);
#pragma unroll 1
        for (int a = 0; a < P; ++a) {
            const T *pl = base - a * W2;
            T sa = T(0), ga = T(0), gza = T(0);
#pragma unroll
            for (int bb = 0; bb < P; ++bb) {
                const T *row = pl - bb * W;
                T sz = T(0), dzs = T(0);
#pragma unroll
                for (int c = 0; c < P; ++c) {
                    const T v = row[-c];
                    sz += cz[c] * v;
                    dzs += dz[c] * v;
                }
                sa += cy[bb] * sz;
                ga += dy[bb] * sz;
                gza += cy[bb] * dzs;
            }
            s += cx[0] * sa;
            gx += dx[0] * sa;
            gy += cx[0] * ga;
            gz += cx[0] * gza;
            shift_down<T, P>(cx, dx);
        }
        const double qk = -(double)pr.w * kl;
        f[3 * (int64_t)slot + 0] = qk * (double)gx;
        f[3 * (int64_t)slot + 1] = qk * (double)gy;
        f[3 * (int64_t)slot + 2] = qk * (double)gz;
        phi[slot] = (double)s;
    }
}

// Host B-spline M_p(u) by the order recursion (for the Euler-spline moduli).
double bspline_host(int p, double u)
{
    if (p == 2) return (u >= 0.0 && u <= 2.0) ? 1.0 - fabs(u - 1.0) : 0.0;
    return u / (p - 1) * bspline_host(p - 1, u) + (p - u) / (p - 1) * bspline_host(p - 1, u - 1.0);
}

cudaError_t upload_axis(Plan &p, SpmeState &s, cudaStream_t st)
{
    const int K = s.K, P = s.order;
    std::vector<double2> ax(K);
    for (int m = 0; m < K; ++m) {
        double re = 0.0, im = 0.0;
        for (int k = 0; k <= P - 2; ++k) {
            const double mk = bspline_host(P, k + 1.0);
            re += mk * cos(2.0 * kPi * m * k / K);
            im += mk * sin(2.0 * kPi * m * k / K);
        }
        const double b2 = 1.0 / (re * re + im * im);
        const double sm = (m <= K / 2 ? m : m - K) / p.L;
        ax[m].x = b2 * exp(-kPi * kPi * sm * sm / (p.beta * p.beta));
        ax[m].y = sm;
    }
    cudaError_t e = cudaMemcpyAsync(s.axis, ax.data(), sizeof(double2) * K, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e == cudaSuccess) { s.axis_beta = p.beta; s.axis_L = p.L; }
    return e;
}

// Tile side (mesh points) of bricks of bc cells per side on an nc-cell grid with K mesh
// points per side and splines of order P: the largest brick's mesh extent plus P + 2.
static int tile_side(int nc, int K, int P, int bc)
{
    int W = 0;
    for (int b = 0; b * bc < nc; ++b) {
        const int c0 = b * bc, c1 = c0 + bc < nc ? c0 + bc : nc;
        const int w = (int)(((int64_t)c1 * K) / nc - ((int64_t)c0 * K) / nc) + P + 2;
        if (w > W) W = w;
    }
    return W;
}

// Brick sizes for the plan's cell grid (bc = 0: no tile fits, e.g. the single cell of a
// small box).  Spreading: the largest bc (cells per brick side, <= 8) whose tile (W <= 40,
// row pitch S = 24 or 40) and chunk fit in half of an SM's shared memory (two blocks per
// SM) while the bricks still fill every SM once; else the largest that fits in one SM's
// shared memory with that many bricks; else the smallest brick that fits.  Gather: the
// smallest bc whose bricks hold >= 128 particles on average (one thread per particle), if
// its tile fits in half of an SM's shared memory and the bricks
// fill the SMs; else the spreading's bricks.  (The gather's tile is W^3 with no padding.)
template <class T, int P>
void choose_tiling(Plan &p, SpmeState &s, int64_t n)
{
    const int nc = p.nc, K = s.K;
    const int chunk = sizeof(T) == 4 ? 128 : 64;
    const size_t max_smem = 227 * 1024 - 1024;
    auto pitch = [](int W) { return W <= 24 ? 24 : 40; };
    auto spread_smem = [&](int W) {
        return (((size_t)W * W * pitch(W) + (size_t)chunk * 3 * P) * sizeof(T) + 7) / 8 * 8 +
               (size_t)chunk * sizeof(int2);
    };
    int pick[3] = {0, 0, 0};
    for (int bc = 1; bc <= 8 && bc <= nc && p.w > 0; ++bc) {
        const int nbk = (nc + bc - 1) / bc;
        const int W = tile_side(nc, K, P, bc);
        if (W > 40 || spread_smem(W) > max_smem) break;
        const bool fill = (int64_t)nbk * nbk * nbk >= p.num_sms;
        if (fill && spread_smem(W) <= max_smem / 2) pick[0] = bc;
        if (fill) pick[1] = bc;
        if (!pick[2]) pick[2] = bc;
    }
    const int bc = pick[0] ? pick[0] : pick[1] ? pick[1] : pick[2];
    s.tile_nc = nc;
    s.bc = bc;
    s.nbk = bc ? (nc + bc - 1) / bc : 0;
    s.W = bc ? tile_side(nc, K, P, bc) : 0;
    s.S = pitch(s.W);
    s.chunk = chunk;
    s.smem = bc ? spread_smem(s.W) : 0;
    s.bc_g = bc;
    for (int g = bc; g >= 1 && g <= 8 && g <= nc; ++g) {
        const int nbk = (nc + g - 1) / g;
        const int W = tile_side(nc, K, P, g);
        if (W > 40 || (size_t)W * W * W * sizeof(T) > max_smem / 2 ||
            (int64_t)nbk * nbk * nbk < p.num_sms)
            break;
        s.bc_g = g;
        if ((double)n / ((double)nbk * nbk * nbk) >= 128.0) break;
    }
    s.nbk_g = s.bc_g ? (nc + s.bc_g - 1) / s.bc_g : 0;
    s.W_g = s.bc_g ? tile_side(nc, K, P, s.bc_g) : 0;
    s.smem_g = (size_t)s.W_g * s.W_g * s.W_g * sizeof(T);
    if (!bc) return;
    size_t cap = 0, cap_g = 0;
    cudaError_t e = s.S == 24 ? smem_optin((const void *)k_spme_spread_tile<T, P, 24>, &cap)
                              : smem_optin((const void *)k_spme_spread_tile<T, P, 40>, &cap);
    if (e == cudaSuccess) e = smem_optin((const void *)k_spme_gather_tile<T, P>, &cap_g);
    if (e == cudaSuccess && (s.smem > cap || s.smem_g > cap_g)) e = cudaErrorInvalidValue;
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        s.bc = s.bc_g = 0;
    }
}

template <class T, int P, int S>
void launch_spread_tile(Plan &p, SpmeState &s, double kl, cudaStream_t st)
{
    k_spme_spread_tile<T, P, S><<<(unsigned)((int64_t)s.nbk * s.nbk * s.nbk), P * 32, s.smem, st>>>(
        p.ws.pg, p.ws.cell_start, p.nc, s.bc, s.nbk, s.W, s.chunk, s.K, kl, s.qfix);
}

template <class T, int P>
void launch_gather_tile(Plan &p, SpmeState &s, double kl, cudaStream_t st)
{
    k_spme_gather_tile<T, P><<<(unsigned)((int64_t)s.nbk_g * s.nbk_g * s.nbk_g), kThreads,
                               s.smem_g, st>>>(
        p.ws.pg, p.ws.cell_start, p.nc, s.bc_g, s.nbk_g, s.W_g, s.K, kl, (const T *)s.mesh,
        p.ws.f_recip, p.ws.phi_recip);
}

template <class T, int P>
cudaError_t launch_spme_p(Plan &p, SpmeState &s, int64_t n, cudaStream_t st)
{
    using T2 = typename std::conditional<sizeof(T) == 4, float2, double2>::type;
    const int K = s.K;
    const int64_t m = (int64_t)K * K * K;
    const double kl = K / p.L;
    const unsigned gb = (unsigned)((n + kThreads - 1) / kThreads);
    prof_mark(p, kEvRecipStart, st);
    if (s.tile_nc != p.nc || s.tile_n != n) choose_tiling<T, P>(p, s, n);
    s.tile_n = n;
    if (s.bc > 0 && s.S == 24) launch_spread_tile<T, P, 24>(p, s, kl, st);
    else if (s.bc > 0) launch_spread_tile<T, P, 40>(p, s, kl, st);
    else
        k_spme_spread<T, P><<<gb, kThreads, 0, st>>>(n, p.ws.pg, K, kl, s.qfix);
    k_spme_convert<T><<<(unsigned)((m + kThreads - 1) / kThreads), kThreads, 0, st>>>(m, s.qfix, (T *)s.mesh);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (cufftSetStream(s.fwd, st) != CUFFT_SUCCESS || cufftSetStream(s.inv, st) != CUFFT_SUCCESS)
        return cudaErrorUnknown;
    cufftResult fr;
    if (sizeof(T) == 4) fr = cufftExecR2C(s.fwd, (cufftReal *)s.mesh, (cufftComplex *)s.spec);
    else fr = cufftExecD2Z(s.fwd, (cufftDoubleReal *)s.mesh, (cufftDoubleComplex *)s.spec);
    if (fr != CUFFT_SUCCESS) return cudaErrorUnknown;
    prof_mark(p, kEvFwdEnd, st);
    const double V = p.L * p.L * p.L;
    k_spme_influence<T, T2><<<s.nblk, kThreads, 0, st>>>(K, s.axis, 1.0 / (kPi * V),
                                                       kPi * kPi / (p.beta * p.beta),
                                                       (T2 *)s.spec, s.part);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    prof_mark(p, kEvCoefEnd, st);
    if (sizeof(T) == 4) fr = cufftExecC2R(s.inv, (cufftComplex *)s.spec, (cufftReal *)s.mesh);
    else fr = cufftExecZ2D(s.inv, (cufftDoubleComplex *)s.spec, (cufftDoubleReal *)s.mesh);
    if (fr != CUFFT_SUCCESS) return cudaErrorUnknown;
    if (s.bc_g > 0) launch_gather_tile<T, P>(p, s, kl, st);
    else
        k_spme_gather<T, P><<<gb, kThreads, 0, st>>>(n, p.ws.pg, K, kl, (const T *)s.mesh,
                                                     p.ws.f_recip, p.ws.phi_recip);
    prof_mark(p, kEvBackEnd, st);
    p.launches += 6;   // 4 kernels + 2 transforms (cuFFT kernels counted as one each)
    return cudaGetLastError();
}

template <class T>
cudaError_t launch_spme_t(Plan &p, SpmeState &s, int64_t n, cudaStream_t st)
{
    switch (s.order) {
        case 4: return launch_spme_p<T, 4>(p, s, n, st);
        case 6: return launch_spme_p<T, 6>(p, s, n, st);
        case 8: return launch_spme_p<T, 8>(p, s, n, st);
        case 10: return launch_spme_p<T, 10>(p, s, n, st);
        case 12: return launch_spme_p<T, 12>(p, s, n, st);
        default: return cudaErrorInvalidValue;
    }
}

void destroy_state(SpmeState *s)
{
    if (!s) return;
    if (s->have_fwd) cufftDestroy(s->fwd);
    if (s->have_inv) cufftDestroy(s->inv);
    cudaFree(s->qfix);
    cudaFree(s->mesh);
    cudaFree(s->spec);
    cudaFree(s->axis);
    cudaFree(s->part);
    delete s;
}

}  // namespace

void spme_free(Plan &p)
{
    destroy_state(static_cast<SpmeState *>(p.spme));
    p.spme = nullptr;
}

int spme_set(Plan &p, int K, int order)
{
    if (K == 0) {
        spme_free(p);
        return EWALD_OK;
    }
    if (order < 4 || order > 12 || (order & 1) || K < order || K > 1024) return EWALD_E_INVAL;
    SpmeState *s = new (std::nothrow) SpmeState();
    if (!s) return EWALD_E_NOMEM;
    s->K = K;
    s->order = order;
    s->fp32 = p.precision != EWALD_FP64;
    const size_t m = (size_t)K * K * K, h = (size_t)K * K * (K / 2 + 1);
    const size_t real = s->fp32 ? sizeof(float) : sizeof(double);
    cudaError_t e = cudaSuccess;
    if (e == cudaSuccess) e = cudaMalloc((void **)&s->qfix, sizeof(unsigned long long) * m);
    if (e == cudaSuccess) e = cudaMalloc(&s->mesh, real * m);
    if (e == cudaSuccess) e = cudaMalloc(&s->spec, 2 * real * h);
    if (e == cudaSuccess) e = cudaMalloc((void **)&s->axis, sizeof(double2) * K);
    s->nblk = 4 * p.num_sms;
    if (e == cudaSuccess) e = cudaMalloc((void **)&s->part, sizeof(double) * 7 * s->nblk);
    if (e == cudaSuccess) e = cudaMemset(s->qfix, 0, sizeof(unsigned long long) * m);
    if (e != cudaSuccess) {
        destroy_state(s);
        return e == cudaErrorMemoryAllocation ? EWALD_E_NOMEM : EWALD_E_CUDA;
    }
    if (cufftPlan3d(&s->fwd, K, K, K, s->fp32 ? CUFFT_R2C : CUFFT_D2Z) != CUFFT_SUCCESS) {
        destroy_state(s);
        return EWALD_E_UNSUPPORTED;
    }
    s->have_fwd = true;
    if (cufftPlan3d(&s->inv, K, K, K, s->fp32 ? CUFFT_C2R : CUFFT_Z2D) != CUFFT_SUCCESS) {
        destroy_state(s);
        return EWALD_E_UNSUPPORTED;
    }
    s->have_inv = true;
    if ((e = upload_axis(p, *s, p.side_stream)) != cudaSuccess) {
        destroy_state(s);
        return EWALD_E_CUDA;
    }
    spme_free(p);
    p.spme = s;
    return EWALD_OK;
}

cudaError_t launch_recip_spme(Plan &p, int64_t n, cudaStream_t st)
{
    SpmeState &s = *static_cast<SpmeState *>(p.spme);
    if (s.axis_beta != p.beta || s.axis_L != p.L) {
        cudaError_t e = upload_axis(p, s, st);
        if (e != cudaSuccess) return e;
    }
    return s.fp32 ? launch_spme_t<float>(p, s, n, st) : launch_spme_t<double>(p, s, n, st);
}

const double *spme_energy_parts(const Plan &p, int *count)
{
    const SpmeState *s = static_cast<const SpmeState *>(p.spme);
    *count = s->nblk;
    return s->part;
}

const double *spme_virial_parts(const Plan &p, int *count)
{
    const SpmeState *s = static_cast<const SpmeState *>(p.spme);
    *count = s->nblk;
    return s->part + s->nblk;
}

size_t spme_bytes(const Plan &p)
{
    const SpmeState *s = static_cast<const SpmeState *>(p.spme);
    if (!s) return 0;
    const size_t K = s->K, m = K * K * K, h = K * K * (K / 2 + 1);
    const size_t real = s->fp32 ? 4 : 8;
    return 8 * m + real * m + 2 * real * h;
}

}  // namespace ew
