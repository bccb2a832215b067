// ewald_real_noalloc: the real-space pair sum for callers that cannot allocate device memory.
//
// Some callers of this library cannot call cudaMalloc (or anything that calls it):
//   * code that runs while a stream is being captured into a CUDA graph, where allocation
//     calls are not allowed;
//   * host programs whose device memory belongs to another allocator (a framework's caching
//     allocator, a memory pool shared with other components) or is capped by a quota;
//   * latency-critical loops that must never enter the driver's allocator.
// The plan-based entry points allocate their workspaces on first use, so they are not usable
// there.  This entry point evaluates the same real-space sum as ewald_compute_async with
// EWALD_PART_REAL (Eq. 4 / Listing 1 of the paper, FP64 arithmetic, every pair with the
// minimum image, forces in the caller's particle order) using only a scratch area that is a
// file-scope __device__ array.  That array is created with the library's device code in every
// GPU context that loads the library and stays there until the process exits; this file never
// calls cudaMalloc or cudaFree.
//
// The scratch holds the packed particles and one energy partial per 32-particle tile, for at
// most EWALD_NOALLOC_MAX_N particles.  All calls share it and it keeps the last call's
// contents; a call overwrites everything it reads before reading it.  Two calls whose work
// overlaps on the GPU (different streams, or the same stream from two host threads without
// ordering) race on the scratch and give undefined results.
//
// In host code the array's name is only a host-side stand-in for the device symbol; its
// device address comes from cudaGetSymbolAddress, looked up on every call with the caller's
// device current (a host-side lookup that allocates nothing), so an address never outlives
// the context it belongs to (after cudaDeviceReset, or for another context on the same
// device).  Every call also asks for the attributes of its three kernels, which makes the
// runtime load them into the context if lazy loading has not done so yet; the first call on
// a device may therefore load the library's device code, and it should come before any
// stream capture.  Each launch is checked by its own return code, so an error left pending
// by some unrelated earlier launch is neither reported as this call's nor cleared.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "ewald_internal.cuh"

namespace {

constexpr int kMaxN = EWALD_NOALLOC_MAX_N;
constexpr int kTile = 32;
constexpr int kTiles = (kMaxN + kTile - 1) / kTile;
constexpr size_t kPackBytes = sizeof(double4_32a) * (size_t)kMaxN;
constexpr size_t kScratchBytes = kPackBytes + sizeof(double) * (size_t)kTiles;

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

// Wrap into [0, L) and pack (x, y, z, q) as FP64.
__global__ void k_na_pack(int n, const double *__restrict__ pos, const double *__restrict__ q,
                          double L, double4_32a *__restrict__ out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double x = pos[3 * i], y = pos[3 * i + 1], z = pos[3 * i + 2];
    x -= L * floor(x / L); if (x >= L) x = 0.0;
    y -= L * floor(y / L); if (y >= L) y = 0.0;
    z -= L * floor(z / L); if (z >= L) z = 0.0;
    out[i] = make_double4_32a(x, y, z, q[i]);
}

// One warp per tile of 32 targets; every lane sums over all partners with the minimum image:
//   F_i = q_i sum_j q_j (r_ij / r_ij^2) [erfc(beta r)/r + 2 beta/sqrt(pi) exp(-beta^2 r^2)],
//   phi_i = sum_j q_j erfc(beta r)/r, pairs with 0 < r < r_c.
__global__ void k_na_pairs(int n, const double4_32a *__restrict__ p, double L, double rc2,
                           double beta, double tbr, double *__restrict__ forces,
                           double *__restrict__ e_tile)
{
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (warp * kTile >= n) return;
    const int i = warp * kTile + lane;
    const bool valid = i < n;
    const double4_32a pi = p[valid ? i : 0];
    const double invL = 1.0 / L;
    double fx = 0.0, fy = 0.0, fz = 0.0, phi = 0.0;
    for (int j = 0; j < n; ++j) {
        const double4_32a pj = p[j];
        double dx = pi.x - pj.x, dy = pi.y - pj.y, dz = pi.z - pj.z;
        dx -= L * rint(dx * invL);
        dy -= L * rint(dy * invL);
        dz -= L * rint(dz * invL);
        const double r2 = dx * dx + dy * dy + dz * dz;
        if (r2 < rc2 && r2 > 0.0) {
            const double r = sqrt(r2);
            const double e = erfc(beta * r) / r;
            const double s = pj.w * (e + tbr * exp(-beta * beta * r2)) / r2;
            phi += pj.w * e;
            fx += s * dx; fy += s * dy; fz += s * dz;
        }
    }
    if (valid) {
        forces[3 * (int64_t)i + 0] = pi.w * fx;
        forces[3 * (int64_t)i + 1] = pi.w * fy;
        forces[3 * (int64_t)i + 2] = pi.w * fz;
    }
    double e = valid ? pi.w * phi : 0.0;
    for (int o = 16; o > 0; o >>= 1) e += __shfl_down_sync(0xffffffffu, e, o);
    if (lane == 0) e_tile[warp] = e;
}

// energy[0] = E_real = 1/2 sum_i q_i phi_i (fixed-order sum), energy[1] = energy[2] = 0,
// energy[3] = E_real.
__global__ void k_na_energy(int ntiles, const double *__restrict__ e_tile,
                            double *__restrict__ energy)
{
    __shared__ double red[256];
    const int t = threadIdx.x;
    double s = 0.0;
    for (int k = t; k < ntiles; k += 256) s += e_tile[k];
    red[t] = s;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (t < o) red[t] += red[t + o];
        __syncthreads();
    }
    if (t == 0) {
        const double er = 0.5 * red[0];
        energy[0] = er;
        energy[1] = 0.0;
        energy[2] = 0.0;
        energy[3] = er;
    }
}

// Launch with the launch's own status (cudaLaunchKernel returns the error of this launch).
template <class T> struct same { using type = T; };
template <class... A>
cudaError_t launch(void (*k)(A...), unsigned grid, unsigned block, cudaStream_t st,
                   typename same<A>::type... a)
{
    void *args[] = {(void *)&a...};
    return cudaLaunchKernel((const void *)k, dim3(grid), dim3(block), args, 0, st);
}

}  // namespace

extern "C" int ewald_real_noalloc(double L, double beta, double r_c, int64_t n, const double *pos,
                                  const double *q, double *forces, double *energy_dev,
                                  void *stream)
{
    if (!(L > 0) || !isfinite(L) || !(beta > 0) || !isfinite(beta)) return EWALD_E_INVAL;
    if (!(r_c > 0) || !(r_c <= 0.5 * L)) return EWALD_E_CUTOFF;
    if (n < 0 || !energy_dev) return EWALD_E_INVAL;
    if (n > kMaxN) return EWALD_E_UNSUPPORTED;
    if (n > 0 && (!pos || !q || !forces)) return EWALD_E_INVAL;
    // every kernel of this entry point is loaded into the current context now, whatever n is
    cudaFuncAttributes fa;
    if (cudaFuncGetAttributes(&fa, k_na_pack) != cudaSuccess ||
        cudaFuncGetAttributes(&fa, k_na_pairs) != cudaSuccess ||
        cudaFuncGetAttributes(&fa, k_na_energy) != cudaSuccess)
        return EWALD_E_CUDA;
    void *base = nullptr;
    if (cudaGetSymbolAddress(&base, g_scratch) != cudaSuccess || !base) return EWALD_E_CUDA;
    cudaStream_t st = (cudaStream_t)stream;
    double4_32a *packed = reinterpret_cast<double4_32a *>(base);
    double *e_tile = reinterpret_cast<double *>(static_cast<unsigned char *>(base) + kPackBytes);
    const int ni = (int)n;
    const int ntiles = (ni + kTile - 1) / kTile;
    if (ni > 0) {
        if (launch(k_na_pack, (unsigned)((ni + 255) / 256), 256u, st, ni, pos, q, L, packed) !=
            cudaSuccess)
            return EWALD_E_CUDA;
        if (launch(k_na_pairs, (unsigned)((ntiles * 32 + 127) / 128), 128u, st, ni,
                   (const double4_32a *)packed, L, r_c * r_c, beta, 2.0 * beta / sqrt(ew::kPi),
                   forces, e_tile) != cudaSuccess)
            return EWALD_E_CUDA;
    }
    if (launch(k_na_energy, 1u, 256u, st, ntiles, (const double *)e_tile, energy_dev) !=
        cudaSuccess)
        return EWALD_E_CUDA;
    return EWALD_OK;
}
