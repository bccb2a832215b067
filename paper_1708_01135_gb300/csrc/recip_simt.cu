// Reciprocal-space sum on CUDA cores (hot-path steps a5-a8), FP64 or FP32 arithmetic.
//
// Section 3.1.2 and Eq. 3 write the long-range potential as two matrix-vector products: an
// N_k x N matrix times the charge vector gives rho_hat_k (Algorithm 1), and an N x N_k
// matrix applied to C_k rho_hat_k gives every particle's potential and force (Algorithm 2).
// Here the k vectors are grouped in rows r = (m_y, m_z) of the half space, with m_x along
// the row, and the phase factors are products of per-axis tables:
//     e^{i k.r_j} = X_j[m_x] Y_j[m_y] Z_j[m_z],  X_j[m] = e^{2 pi i m x_j / L}  (same for y, z)
// computed once per particle by an FP64 recurrence X_j[m] = X_j[m-1] e^{2 pi i x_j / L}.
//
// Step a6 (structure factors, forward product).  With A_j[r] = q_j Y_j[m_y] Z_j[m_z]:
//     T_ab[r, m] = sum_j a(A_j[r]) b(X_j[m]),  a, b in {Re, Im},  m = 0..k_max
//     S[r, +m] = (T_rr - T_ii) + i (T_ri + T_ir),   S[r, -m] = (T_rr + T_ii) + i (T_ir - T_ri)
// (X_j[-m] = conj X_j[m], so the four real sums for m >= 0 give both signs of m_x).
//
// Step a7 (energy, coefficients).  g(k) = 4 pi exp(-k^2 / (4 beta^2)) / (V k^2) (C_k of Eq. 3)
//     E_recip = sum_{k in K_half} g(k) |S(k)|^2        G(k) = 2 g(k) conj S(k)
//
// Step a8 (back-scatter, Algorithm 2).  With P_i[r] = Y_i[m_y] Z_i[m_z] and
// U_i[m] = sum_r P_i[r] G[r, m] (complex), the force and potential of particle i are
//     F_x = q_i (2 pi / L) sum_m m Im(X_i[m] U_i[m]),   F_y, F_z likewise with U^y, U^z
//     (G weighted by m_y or m_z),   phi_i = sum_m Re(X_i[m] U_i[m]).
// Pairing m with -m leaves, per component block, 2 k_max + 1 real columns of a real matrix
// G' [2R x 3(2 k_max + 1)] (rows: Re P, Im P of every row r) - the second product is the
// real matrix product [Re P, Im P] G' followed by a short per-particle sum over m >= 0.
// Column c of a block: c = 0 is the m = 0 term; c = 2m - 1 and c = 2m are the two
// combinations of +m and -m needed with Re X_i[m] and Im X_i[m]:
//   block x: c0 = Re U[0];  D1[m] = Im(U[m] - U[-m]),  D2[m] = Re(U[m] + U[-m])
//            F_x ~ sum_m m (Re X[m] D1[m] + Im X[m] D2[m]),
//            phi = Re U[0] + sum_m (Re X[m] D2[m] - Im X[m] D1[m])
//   block y: c0 = Im U^y[0];  E1[m] = Im(U^y[m] + U^y[-m]),  E2[m] = Re(U^y[m] - U^y[-m])
//            F_y ~ Im U^y[0] + sum_m (Re X[m] E1[m] + Im X[m] E2[m])     (block z alike)
#include <cuda_runtime.h>
#include <stdint.h>

#include "ewald_internal.cuh"

namespace ew {
namespace {

template <class T> struct Cplx;
template <> struct Cplx<float> { using type = float2; };
template <> struct Cplx<double> { using type = double2; };

constexpr int kRT = 32;       // rows per forward block
constexpr int kPC = 32;       // particles per forward chunk
constexpr int kNV = 4;        // m values per thread in the forward block (8 warps x 4 = 32)
constexpr int kBP = 64;       // particles per back-scatter block
constexpr int kBC = 64;       // columns per back-scatter pass (4 groups x 16)
constexpr int kBK = 16;       // rows per back-scatter chunk (32 real K)

// a5: per-axis phase tables by FP64 recurrence from the FP64 base phase.
template <class T>
__global__ void k_tables(int64_t n, int64_t cap, const double4_32a *__restrict__ pg, double L,
                         int kmax, typename Cplx<T>::type *__restrict__ X,
                         typename Cplx<T>::type *__restrict__ Y,
                         typename Cplx<T>::type *__restrict__ Z)
{
    using C = typename Cplx<T>::type;
    int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    const double4_32a p = pg[s];
    const double a[3] = {p.x, p.y, p.z};
    for (int ax = 0; ax < 3; ++ax) {
        double bs, bc;
        sincospi(2.0 * a[ax] / L, &bs, &bc);
        double cr = 1.0, ci = 0.0;
        for (int m = 0; m <= kmax; ++m) {
            C v;
            v.x = (T)cr;
            v.y = (T)ci;
            if (ax == 0) X[(int64_t)m * cap + s] = v;
            else if (ax == 1) {
                Y[(int64_t)(kmax + m) * cap + s] = v;
                C w; w.x = v.x; w.y = -v.y;
                Y[(int64_t)(kmax - m) * cap + s] = w;
            } else Z[(int64_t)m * cap + s] = v;
            double nr = cr * bc - ci * bs;
            double ni = cr * bs + ci * bc;
            cr = nr;
            ci = ni;
        }
    }
}

// a6: forward product, partial sums over a slice of particles.
// grid (row tiles, K splits, m chunks of 32); block 256 threads.
template <class T>
__global__ void __launch_bounds__(256)
k_sfac(int64_t n, int64_t cap, int nks, int R, int kmax, const RowInfo *__restrict__ rows,
       const double4_32a *__restrict__ pg, const typename Cplx<T>::type *__restrict__ X,
       const typename Cplx<T>::type *__restrict__ Y, const typename Cplx<T>::type *__restrict__ Z,
       T *__restrict__ spart)
{
    using C = typename Cplx<T>::type;
    __shared__ C As[kPC][kRT];
    __shared__ C Xs[kPC][kNV * 8];
    const int t = threadIdx.x, lane = t & 31, g = t >> 5;
    const int r0 = blockIdx.x * kRT;
    const int ks = blockIdx.y;
    const int m0 = blockIdx.z * kNV * 8;
    const int64_t per = (n + nks - 1) / nks;
    const int64_t p0 = ks * per;
    const int64_t p1 = p0 + per < n ? p0 + per : n;
    T acc[kNV][4];
#pragma unroll
    for (int v = 0; v < kNV; ++v) acc[v][0] = acc[v][1] = acc[v][2] = acc[v][3] = T(0);
    for (int64_t pc = p0; pc < p1; pc += kPC) {
        for (int e = t; e < kPC * kRT; e += 256) {
            const int j = e % kPC, rl = e / kPC;
            const int64_t s = pc + j;
            C a; a.x = T(0); a.y = T(0);
            if (s < p1 && r0 + rl < R) {
                const RowInfo ri = rows[r0 + rl];
                const C y = Y[(int64_t)(kmax + ri.my) * cap + s];
                const C z = Z[(int64_t)ri.mz * cap + s];
                const T q = (T)pg[s].w;
                a.x = q * (y.x * z.x - y.y * z.y);
                a.y = q * (y.x * z.y + y.y * z.x);
            }
            As[j][rl] = a;
        }
        for (int e = t; e < kPC * kNV * 8; e += 256) {
            const int j = e % kPC, ml = e / kPC;
            const int64_t s = pc + j;
            C x; x.x = T(0); x.y = T(0);
            if (s < p1 && m0 + ml <= kmax) x = X[(int64_t)(m0 + ml) * cap + s];
            Xs[j][ml] = x;
        }
        __syncthreads();
#pragma unroll 4
        for (int j = 0; j < kPC; ++j) {
            const C a = As[j][lane];
#pragma unroll
            for (int v = 0; v < kNV; ++v) {
                const C x = Xs[j][g + 8 * v];
                acc[v][0] += a.x * x.x;   // T_rr
                acc[v][1] += a.x * x.y;   // T_ri
                acc[v][2] += a.y * x.x;   // T_ir
                acc[v][3] += a.y * x.y;   // T_ii
            }
        }
        __syncthreads();
    }
    const int r = r0 + lane;
    if (r >= R) return;
#pragma unroll
    for (int v = 0; v < kNV; ++v) {
        const int m = m0 + g + 8 * v;
        if (m > kmax) continue;
        T *o = spart + (((int64_t)ks * R + r) * (kmax + 1) + m) * 4;
        o[0] = acc[v][0]; o[1] = acc[v][1]; o[2] = acc[v][2]; o[3] = acc[v][3];
    }
}

// a6 (reduction over K splits, fixed order) + a7 (per-k energy, coefficient matrix).
// One block per row, thread m = 0..kmax.
template <class T>
__global__ void k_sreduce(int nks, int R, int kmax, const RowInfo *__restrict__ rows,
                          const T *__restrict__ spart, const double *__restrict__ gk,
                          double *__restrict__ S, double *__restrict__ e_row,
                          T *__restrict__ gmat, int ncol)
{
    __shared__ double red[128];
    const int r = blockIdx.x, m = threadIdx.x;
    const RowInfo ri = rows[r];
    double e = 0.0;
    const int nb = 2 * kmax + 1;
    if (m <= kmax) {
        double t[4] = {0.0, 0.0, 0.0, 0.0};
        for (int ks = 0; ks < nks; ++ks) {
            const T *o = spart + (((int64_t)ks * R + r) * (kmax + 1) + m) * 4;
            t[0] += (double)o[0]; t[1] += (double)o[1]; t[2] += (double)o[2]; t[3] += (double)o[3];
        }
        const bool origin_row = (ri.my == 0 && ri.mz == 0);
        const bool vp = m <= ri.nxmax && (!origin_row || m > 0);           // mode (+m, my, mz)
        const bool vn = m >= 1 && m <= ri.nxmax && !origin_row;           // mode (-m, my, mz)
        double spr = t[0] - t[3], spi = t[2] + t[1];                      // S(+m)
        double snr = t[0] + t[3], sni = t[2] - t[1];                      // S(-m)
        double gp = 0.0, gn = 0.0;
        if (vp) {
            int idx = origin_row ? ri.koff + (m - 1) : ri.koff + ri.nxmax + m;
            gp = gk[idx];
            S[2 * (int64_t)idx] = spr; S[2 * (int64_t)idx + 1] = spi;
            e += gp * (spr * spr + spi * spi);
        }
        if (vn && m > 0) {
            int idx = ri.koff + ri.nxmax - m;
            gn = gk[idx];
            S[2 * (int64_t)idx] = snr; S[2 * (int64_t)idx + 1] = sni;
            e += gn * (snr * snr + sni * sni);
        }
        // G = 2 g conj(S): Gr = 2 g Sr, Gi = -2 g Si (zero outside K_half)
        const double Gpr = vp ? 2.0 * gp * spr : 0.0, Gpi = vp ? -2.0 * gp * spi : 0.0;
        const double Gnr = vn ? 2.0 * gn * snr : 0.0, Gni = vn ? -2.0 * gn * sni : 0.0;
        T *row_re = gmat + (int64_t)(2 * r) * ncol;
        T *row_im = gmat + (int64_t)(2 * r + 1) * ncol;
        const double wy = (double)ri.my, wz = (double)ri.mz;
        if (m == 0) {
            row_re[0] = (T)Gpr;            row_im[0] = (T)(-Gpi);               // Re U[0]
            row_re[nb] = (T)(wy * Gpi);    row_im[nb] = (T)(wy * Gpr);          // Im U^y[0]
            row_re[2 * nb] = (T)(wz * Gpi); row_im[2 * nb] = (T)(wz * Gpr);     // Im U^z[0]
        } else {
            const int c1 = 2 * m - 1, c2 = 2 * m;
            // block x: D1 = Im(U[m] - U[-m]), D2 = Re(U[m] + U[-m])
            row_re[c1] = (T)(Gpi - Gni);   row_im[c1] = (T)(Gpr - Gnr);
            row_re[c2] = (T)(Gpr + Gnr);   row_im[c2] = (T)(-(Gpi + Gni));
            // blocks y, z: E1 = Im(U^w[m] + U^w[-m]), E2 = Re(U^w[m] - U^w[-m])
            row_re[nb + c1] = (T)(wy * (Gpi + Gni));      row_im[nb + c1] = (T)(wy * (Gpr + Gnr));
            row_re[nb + c2] = (T)(wy * (Gpr - Gnr));      row_im[nb + c2] = (T)(-wy * (Gpi - Gni));
            row_re[2 * nb + c1] = (T)(wz * (Gpi + Gni));  row_im[2 * nb + c1] = (T)(wz * (Gpr + Gnr));
            row_re[2 * nb + c2] = (T)(wz * (Gpr - Gnr));  row_im[2 * nb + c2] = (T)(-wz * (Gpi - Gni));
        }
    }
    // zero the padding columns of this row pair
    for (int c = 3 * nb + m; c < ncol; c += blockDim.x) {
        gmat[(int64_t)(2 * r) * ncol + c] = T(0);
        gmat[(int64_t)(2 * r + 1) * ncol + c] = T(0);
    }
    red[m] = e;
    __syncthreads();
    for (int o = 64; o > 0; o >>= 1) {
        if (m < o) red[m] += red[m + o];
        __syncthreads();
    }
    if (m == 0) e_row[r] = red[0];
}

// a8: back-scatter product [Re P, Im P] G' for 64 particles x one pass of 64 columns of one
// component block, then the per-particle sum over m.  grid (particle tiles, 3 blocks, passes).
// Writes out[((blk * npass + pass) * n + s) * 2 + {0: force part, 1: phi part}].
template <class T>
__global__ void __launch_bounds__(256)
k_bscat(int64_t n, int64_t cap, int R, int kmax, int ncol, int npass,
        const RowInfo *__restrict__ rows, const typename Cplx<T>::type *__restrict__ X,
        const typename Cplx<T>::type *__restrict__ Y, const typename Cplx<T>::type *__restrict__ Z,
        const T *__restrict__ gmat, double *__restrict__ out)
{
    using C = typename Cplx<T>::type;
    __shared__ T Ps[2 * kBK][kBP];
    __shared__ T Gs[2 * kBK][kBC];
    __shared__ double red[4][kBP][2];
    const int t = threadIdx.x, p = t % kBP, cg = t / kBP;
    const int64_t s0 = (int64_t)blockIdx.x * kBP;
    const int blk = blockIdx.y, pass = blockIdx.z;
    const int nb = 2 * kmax + 1;
    const int c0 = blk * nb + pass * kBC;           // first column of this pass in G'
    const int cmax = nb - pass * kBC;               // columns of the block left in this pass
    T acc[kBC / 4];
#pragma unroll
    for (int c = 0; c < kBC / 4; ++c) acc[c] = T(0);
    for (int r0 = 0; r0 < R; r0 += kBK) {
        for (int e = t; e < kBK * kBP; e += 256) {
            const int pl = e % kBP, rl = e / kBP;
            const int64_t s = s0 + pl;
            T re = T(0), im = T(0);
            if (s < n && r0 + rl < R) {
                const RowInfo ri = rows[r0 + rl];
                const C y = Y[(int64_t)(kmax + ri.my) * cap + s];
                const C z = Z[(int64_t)ri.mz * cap + s];
                re = y.x * z.x - y.y * z.y;
                im = y.x * z.y + y.y * z.x;
            }
            Ps[2 * rl][pl] = re;
            Ps[2 * rl + 1][pl] = im;
        }
        for (int e = t; e < 2 * kBK * kBC; e += 256) {
            const int cl = e % kBC, kl = e / kBC;
            const int rr = 2 * r0 + kl;
            T v = T(0);
            if (rr < 2 * R && cl < cmax) v = gmat[(int64_t)rr * ncol + c0 + cl];
            Gs[kl][cl] = v;
        }
        __syncthreads();
#pragma unroll 4
        for (int kk = 0; kk < 2 * kBK; ++kk) {
            const T a = Ps[kk][p];
#pragma unroll
            for (int c = 0; c < kBC / 4; ++c) acc[c] += a * Gs[kk][cg + 4 * c];
        }
        __syncthreads();
    }
    // epilogue: combine with X_i[m]
    const int64_t s = s0 + p;
    double fsum = 0.0, psum = 0.0;
    if (s < n) {
#pragma unroll
        for (int c = 0; c < kBC / 4; ++c) {
            const int col = pass * kBC + cg + 4 * c;   // column within the block
            if (col >= nb) continue;
            const double v = (double)acc[c];
            if (col == 0) {
                if (blk == 0) psum += v; else fsum += v;
                continue;
            }
            const int m = (col + 1) / 2;
            const C x = X[(int64_t)m * cap + s];
            const double xr = (double)x.x, xi = (double)x.y;
            const bool first = (col & 1) == 1;           // D1/E1 (odd) or D2/E2 (even)
            if (blk == 0) {
                fsum += m * (first ? xr * v : xi * v);
                psum += first ? -xi * v : xr * v;
            } else {
                fsum += first ? xr * v : xi * v;
            }
        }
    }
    red[cg][p][0] = fsum;
    red[cg][p][1] = psum;
    __syncthreads();
    if (cg == 0 && s < n) {
        double f = red[0][p][0] + red[1][p][0] + red[2][p][0] + red[3][p][0];
        double ph = red[0][p][1] + red[1][p][1] + red[2][p][1] + red[3][p][1];
        double *o = out + (((int64_t)blk * npass + pass) * n + s) * 2;
        o[0] = f;
        o[1] = ph;
    }
}

// Sum the passes (fixed order) into the sorted reciprocal forces.
__global__ void k_bscat_sum(int64_t n, int npass, const double *__restrict__ part,
                            const double4_32a *__restrict__ pg, double L, double *__restrict__ f,
                            double *__restrict__ phi)
{
    int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    const double qf = pg[s].w * (2.0 * kPi / L);
    for (int blk = 0; blk < 3; ++blk) {
        double v = 0.0;
        for (int ps = 0; ps < npass; ++ps) v += part[(((int64_t)blk * npass + ps) * n + s) * 2];
        f[3 * s + blk] = qf * v;
    }
    // the potential is carried by the x block (phi = Re U[0] + sum_m (...))
    double v = 0.0;
    for (int ps = 0; ps < npass; ++ps) v += part[((int64_t)ps * n + s) * 2 + 1];
    phi[s] = v;
}

int bscat_passes(int kmax) { return (2 * kmax + 1 + kBC - 1) / kBC; }
int forward_splits(const Plan &p, int64_t n)
{
    // enough blocks to fill the GPU: row tiles x m chunks x splits >= ~600
    int tiles = (p.R + kRT - 1) / kRT;
    int mch = (p.kmax + 1 + kNV * 8 - 1) / (kNV * 8);
    int want = (600 + tiles * mch - 1) / (tiles * mch);
    int64_t maxs = (n + 255) / 256;
    if (want > maxs) want = (int)maxs;
    return want < 1 ? 1 : want;
}

template <class T>
cudaError_t launch_t(Plan &p, int64_t n, cudaStream_t st)
{
    using C = typename Cplx<T>::type;
    Workspace &ws = p.ws;
    const int64_t cap = ws.cap_n;
    C *X = (C *)ws.tabX, *Y = (C *)ws.tabY, *Z = (C *)ws.tabZ;
    prof_mark(p, kEvRecipStart, st);
    k_tables<T><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, cap, ws.pg, p.L, p.kmax, X, Y, Z);
    const int nks = forward_splits(p, n);
    dim3 gf((p.R + kRT - 1) / kRT, nks, (p.kmax + 1 + kNV * 8 - 1) / (kNV * 8));
    k_sfac<T><<<gf, 256, 0, st>>>(n, cap, nks, p.R, p.kmax, p.rows_d, ws.pg, X, Y, Z,
                                  (T *)ws.spart);
    prof_mark(p, kEvFwdEnd, st);
    const int nb = 2 * p.kmax + 1;
    const int ncol = 3 * nb;
    k_sreduce<T><<<p.R, 128, 0, st>>>(nks, p.R, p.kmax, p.rows_d, (const T *)ws.spart, p.g_d,
                                      p.S_d, p.e_recip_part, (T *)ws.gmat, ncol);
    prof_mark(p, kEvCoefEnd, st);
    const int npass = bscat_passes(p.kmax);
    dim3 gb((unsigned)((n + kBP - 1) / kBP), 3, npass);
    // the second half of the partials buffer holds the back-scatter pass sums
    double *part = reinterpret_cast<double *>(reinterpret_cast<char *>(ws.spart) + ws.spart_bytes / 2);
    prof_mark(p, kEvBsStart, st);
    k_bscat<T><<<gb, 256, 0, st>>>(n, cap, p.R, p.kmax, ncol, npass, p.rows_d, X, Y, Z,
                                   (const T *)ws.gmat, part);
    prof_mark(p, kEvBsEnd, st);
    p.prof_bs = p.prof;
    k_bscat_sum<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, npass, part, ws.pg, p.L,
                                                             ws.f_recip, ws.phi_recip);
    prof_mark(p, kEvBackEnd, st);
    p.launches += 5;
    return cudaGetLastError();
}

}  // namespace

size_t recip_simt_bytes(const Plan &p, int64_t n)
{
    const size_t es = p.precision == EWALD_FP64 ? 8 : 4;
    const size_t tab = (size_t)n * (size_t)(4 * p.kmax + 3) * 2 * es;
    const int nks = forward_splits(p, n);
    const size_t sp = (size_t)nks * p.R * (p.kmax + 1) * 4 * es;
    const size_t bp = (size_t)3 * bscat_passes(p.kmax) * n * 2 * sizeof(double);
    const size_t gm = (size_t)2 * p.R * 3 * (2 * p.kmax + 1) * es;
    return tab + 2 * (sp > bp ? sp : bp) + gm;
}

cudaError_t alloc_recip_simt(Plan &p, int64_t n)
{
    free_recip_simt(p);
    Workspace &ws = p.ws;
    const size_t es = p.precision == EWALD_FP64 ? 8 : 4;
    const size_t ce = 2 * es;
    cudaError_t e;
    cudaStream_t st = p.side_stream;
    if ((e = pool_alloc(&ws.tabX, (size_t)n * (p.kmax + 1) * ce, st)) != cudaSuccess) return e;
    if ((e = pool_alloc(&ws.tabY, (size_t)n * (2 * p.kmax + 1) * ce, st)) != cudaSuccess) return e;
    if ((e = pool_alloc(&ws.tabZ, (size_t)n * (p.kmax + 1) * ce, st)) != cudaSuccess) return e;
    const int nks = forward_splits(p, n);
    const size_t sp = (size_t)nks * p.R * (p.kmax + 1) * 4 * es;
    const size_t bp = (size_t)3 * bscat_passes(p.kmax) * n * 2 * sizeof(double);
    ws.spart_bytes = 2 * (sp > bp ? sp : bp);
    if ((e = pool_alloc(&ws.spart, ws.spart_bytes, st)) != cudaSuccess) return e;
    ws.gmat_bytes = (size_t)2 * p.R * 3 * (2 * p.kmax + 1) * es;
    if ((e = pool_alloc(&ws.gmat, ws.gmat_bytes, st)) != cudaSuccess) return e;
    return cudaSuccess;
}

void free_recip_simt(Plan &p)
{
    Workspace &ws = p.ws;
    pool_free(ws.tabX, p.side_stream); pool_free(ws.tabY, p.side_stream);
    pool_free(ws.tabZ, p.side_stream); pool_free(ws.spart, p.side_stream);
    pool_free(ws.gmat, p.side_stream);
    ws.tabX = ws.tabY = ws.tabZ = ws.spart = ws.gmat = nullptr;
    ws.spart_bytes = ws.gmat_bytes = 0;
}

cudaError_t launch_recip_simt(Plan &p, int64_t n, cudaStream_t st)
{
    if (p.precision == EWALD_FP64) return launch_t<double>(p, n, st);
    return launch_t<float>(p, n, st);
}

}  // namespace ew
