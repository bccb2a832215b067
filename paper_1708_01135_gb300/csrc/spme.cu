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
//   * spread: one thread per (sorted) particle computes its 3 x p spline weights and adds
//     q w_x w_y w_z to the p^3 mesh points with 64-bit integer atomics on a fixed-point mesh
//     (2^-36 resolution).  Integer addition is associative, so the mesh, and everything
//     after it, is bit-identical from run to run whatever order the atomics land in;
//   * convert (fixed point -> FP64/FP32, and re-zero the fixed-point mesh for the next call),
//     cuFFT real-to-complex transform (a plain library FFT);
//   * influence: G is the product of three per-axis tables and 1 / |m~|^2, computed on the
//     fly (no K^3 coefficient array); the same pass forms the energy and virial partials
//     (fixed-order block sums) and scales the spectrum by G;
//   * cuFFT complex-to-real transform, then gather: one thread per particle reads its p^3
//     mesh values and writes its own force and potential (no atomics).
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
    double *epart = nullptr;              // [kVirBlocks] energy partials
    double axis_beta = 0, axis_L = 0;     // parameters the axis table was built for
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

template <class T, int P>
__global__ void __launch_bounds__(kThreads)
k_spme_spread(int64_t n, const double4_32a *__restrict__ pg, int K, double kl,
              unsigned long long *__restrict__ qfix)
{
    const int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x;
    if (i >= n) return;
    const double4_32a r = pg[i];
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
// for their conjugate partners) and spec <- G spec.  Block b takes the entries
// b * 256 + t + j * (gridDim.x * 256) in order, then a fixed tree.
template <class T2>
__global__ void __launch_bounds__(kThreads)
k_spme_influence(int K, const double2 *__restrict__ axis, double inv_piV, double pi2_b2,
                 T2 *__restrict__ spec, double *__restrict__ epart, double *__restrict__ vpart)
{
    __shared__ double red[7][kThreads];
    const int Kh = K / 2 + 1;
    const int64_t tot = (int64_t)K * K * Kh;
    const int t = threadIdx.x;
    double acc[7] = {0, 0, 0, 0, 0, 0, 0};
    for (int64_t e = (int64_t)blockIdx.x * kThreads + t; e < tot; e += (int64_t)gridDim.x * kThreads) {
        const int mz = (int)(e % Kh);
        const int64_t r = e / Kh;
        const int my = (int)(r % K), mx = (int)(r / K);
        const double2 ax = axis[mx], ay = axis[my], az = axis[mz];
        const double m2 = ax.y * ax.y + ay.y * ay.y + az.y * az.y;
        const double G = e == 0 ? 0.0 : ax.x * ay.x * az.x * inv_piV / m2;
        T2 v = spec[e];
        const double a = G * ((double)v.x * (double)v.x + (double)v.y * (double)v.y);
        const bool single = mz == 0 || 2 * mz == K;    // stands for itself only
        const double hw = single ? 0.5 * a : a;         // 1/2 x (1 or 2)
        if (e != 0) {
            const double c = 2.0 * (1.0 / m2 + pi2_b2);
            // an entry that also stands for its conjugate partner (-m): the partner's signed
            // frequencies are -s, except on a Nyquist index K/2, which is +K/2 for both
            // (the mesh cannot tell +K/2 from -K/2), so there the off-diagonal products of
            // the pair cancel
            const bool nx = 2 * mx == K, ny = 2 * my == K;
            const double fxy = (!single && nx != ny) ? 0.0 : 1.0;
            const double fxz = (!single && nx) ? 0.0 : 1.0, fyz = (!single && ny) ? 0.0 : 1.0;
            acc[0] += hw;
            acc[1] += hw * (1.0 - c * ax.y * ax.y);
            acc[2] += hw * (1.0 - c * ay.y * ay.y);
            acc[3] += hw * (1.0 - c * az.y * az.y);
            acc[4] -= fxy * hw * c * ax.y * ay.y;
            acc[5] -= fxz * hw * c * ax.y * az.y;
            acc[6] -= fyz * hw * c * ay.y * az.y;
        }
        v.x = (decltype(v.x))((double)v.x * G);
        v.y = (decltype(v.y))((double)v.y * G);
        spec[e] = v;
    }
#pragma unroll
    for (int c = 0; c < 7; ++c) red[c][t] = acc[c];
    __syncthreads();
    for (int o = kThreads / 2; o > 0; o >>= 1) {
        if (t < o) {
#pragma unroll
            for (int c = 0; c < 7; ++c) red[c][t] += red[c][t + o];
        }
        __syncthreads();
    }
    if (t == 0) epart[blockIdx.x] = red[0][0];
    if (t < 6) vpart[t * gridDim.x + blockIdx.x] = red[1 + t][0];
}

template <class T, int P>
__global__ void __launch_bounds__(kThreads)
k_spme_gather(int64_t n, const double4_32a *__restrict__ pg, int K, double kl,
              const T *__restrict__ mesh, double *__restrict__ f, double *__restrict__ phi)
{
    const int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x;
    if (i >= n) return;
    const double4_32a r = pg[i];
    int b[3];
    double w[3];
    axis_pos(r.x, kl, K, b[0], w[0]);
    axis_pos(r.y, kl, K, b[1], w[1]);
    axis_pos(r.z, kl, K, b[2], w[2]);
    T cx[P], cy[P], cz[P], dx[P], dy[P], dz[P];
    spline<T, P, true>((T)w[0], cx, dx);
    spline<T, P, true>((T)w[1], cy, dy);
    spline<T, P, true>((T)w[2], cz, dz);
    int iz[P];
#pragma unroll
    for (int c = 0; c < P; ++c) iz[c] = b[2] - c < 0 ? b[2] - c + K : b[2] - c;
    T s = T(0), gx = T(0), gy = T(0), gz = T(0);
#pragma unroll 1
    for (int a = 0; a < P; ++a) {
        const int ix = b[0] - a < 0 ? b[0] - a + K : b[0] - a;
        T sa = T(0), ga = T(0), gza = T(0);
#pragma unroll 1
        for (int bb = 0; bb < P; ++bb) {
            const int iy = b[1] - bb < 0 ? b[1] - bb + K : b[1] - bb;
            const T *row = mesh + ((int64_t)ix * K + iy) * K;
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
        s += cx[a] * sa;
        gx += dx[a] * sa;
        gy += cx[a] * ga;
        gz += cx[a] * gza;
    }
    const double qk = -(double)r.w * kl;
    f[3 * i + 0] = qk * (double)gx;
    f[3 * i + 1] = qk * (double)gy;
    f[3 * i + 2] = qk * (double)gz;
    phi[i] = (double)s;
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

template <class T, int P>
cudaError_t launch_spme_p(Plan &p, SpmeState &s, int64_t n, cudaStream_t st)
{
    using T2 = typename std::conditional<sizeof(T) == 4, float2, double2>::type;
    const int K = s.K;
    const int64_t m = (int64_t)K * K * K;
    const double kl = K / p.L;
    const unsigned gb = (unsigned)((n + kThreads - 1) / kThreads);
    prof_mark(p, kEvRecipStart, st);
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
    k_spme_influence<T2><<<kVirBlocks, kThreads, 0, st>>>(K, s.axis, 1.0 / (kPi * V),
                                                        kPi * kPi / (p.beta * p.beta),
                                                        (T2 *)s.spec, s.epart, p.ws.vir_part);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    prof_mark(p, kEvCoefEnd, st);
    if (sizeof(T) == 4) fr = cufftExecC2R(s.inv, (cufftComplex *)s.spec, (cufftReal *)s.mesh);
    else fr = cufftExecZ2D(s.inv, (cufftDoubleComplex *)s.spec, (cufftDoubleReal *)s.mesh);
    if (fr != CUFFT_SUCCESS) return cudaErrorUnknown;
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
    cudaFree(s->epart);
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
    if (e == cudaSuccess) e = cudaMalloc((void **)&s->epart, sizeof(double) * kVirBlocks);
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
    *count = kVirBlocks;
    return static_cast<const SpmeState *>(p.spme)->epart;
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
